"""The constant-time (bitsliced) cipher's code, run on the host through its
test hook, against the oracle: every key size, both directions, partial
32-block groups.  The circuit's S-box, inverse S-box and InvMixColumns
factoring are also checked at compile time (static_asserts)."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_bitsliced_host_matches_oracle(orc, keybits):
    for seed in range(3):
        key = wl.random_key(keybits, 200 + seed).tobytes()
        enc, dec, nr = aesgb.aes_expand_key(keybits, key)
        for n in (1, 31, 32, 33, 96):
            data = wl.random_bytes(16 * n, 300 + n + seed)
            ct = aesgb.aes_ct_selftest_host(0, enc, nr, data)
            assert np.array_equal(ct, orc.ecb(0, key, data)), (seed, n)
            pt = aesgb.aes_ct_selftest_host(1, dec, nr, ct)
            assert np.array_equal(pt, data), (seed, n)


def test_bitsliced_host_identical_blocks(orc):
    key = wl.random_key(128, 210).tobytes()
    enc, _, nr = aesgb.aes_expand_key(128, key)
    data = np.zeros(16 * 64, np.uint8)
    ct = aesgb.aes_ct_selftest_host(0, enc, nr, data).reshape(-1, 16)
    assert (ct == ct[0]).all()
    assert np.array_equal(ct[0], orc.ecb(0, key, np.zeros(16, np.uint8)))
