"""The constant-time (bitsliced) cipher's code, run on the host through its
test hook, against the oracle: every key size, both directions, partial
32-block groups.  The generated circuits (S-box, inverse S-box core and
output, MixColumns, InvMixColumns with the S-box output map) are also checked
at compile time (static_asserts in bitslice.cuh)."""
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


def test_generated_circuits_are_fresh():
    """bitslice_circuits.h is exactly what gen_bitslice.py writes (the
    generator also re-verifies every circuit against the S-box, the inverse
    S-box, MixColumns and InvMixColumns before writing)."""
    import subprocess
    import sys
    from pathlib import Path
    gen = Path(aesgb.__file__).resolve().parent / "csrc" / "gen_bitslice.py"
    r = subprocess.run([sys.executable, str(gen), "--check"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
