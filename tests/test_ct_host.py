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


def test_ops_per_block_counts_the_circuits():
    """aes_ct_ops_per_block is the gate count of what one block goes through
    (the generated tables' sizes, as the header's comments state them)."""
    import re
    from pathlib import Path
    hdr = (Path(aesgb.__file__).resolve().parent / "csrc" / "bitslice_circuits.h").read_text()
    gates = {name: int(n) for name, n in re.findall(r"// (\w+): \d+ inputs, (\d+) gates", hdr)}
    assert set(gates) == {"sbox_enc", "sbox_core_dec", "sbox_out_dec", "inv_mix_out", "mix_columns"}
    fixed = 128 + 8 * 160  # step-0 key planes, 8 transposes of 32 words
    for nr in (10, 12, 14):
        enc = fixed + 16 * nr * gates["sbox_enc"] + 4 * (nr - 1) * gates["mix_columns"]
        dec = (fixed + 16 * nr * gates["sbox_core_dec"] + 4 * (nr - 1) * gates["inv_mix_out"]
               + 16 * gates["sbox_out_dec"])
        assert aesgb.aes_ct_ops_per_block(0, nr) == enc / 32
        assert aesgb.aes_ct_ops_per_block(1, nr) == dec / 32
    with pytest.raises(aesgb.AesError):
        aesgb.aes_ct_ops_per_block(0, 11)
    with pytest.raises(aesgb.AesError):
        aesgb.aes_ct_ops_per_block(2, 10)
