"""Constant-time (bitsliced) ECB on the GPU: bit-exact against the oracle
for every key size and direction, ragged sizes that leave partial 32-block
groups and partial warp chunks, and equal to the T-table path on a larger
buffer."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_ct_matches_oracle(orc, keybits):
    torch = torch_cuda()
    key = wl.random_key(keybits, 220).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    for n in (1, 31, 32, 33, 1023, 1025, 70_001):
        data = wl.random_bytes(16 * n, 221 + n)
        x = torch.from_numpy(data).cuda()
        y = torch.full((16 * n + 64,), 0x5A, dtype=torch.uint8, device="cuda")
        aesgb.aes_ecb_crypt_ct(0, enc, nr, x, y, n)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.array_equal(got[:16 * n], orc.ecb(0, key, data, nthreads=8)), n
        assert np.all(got[16 * n:] == 0x5A)
        aesgb.aes_ecb_crypt_ct(1, dec, nr, y, y, n)       # in place
        torch.cuda.synchronize()
        assert torch.equal(y[:16 * n], x), n


def test_ct_equals_table_path():
    torch = torch_cuda()
    n = 1 << 22                                         # 64 MiB
    x = torch.empty(16 * n, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.BASE_SEED + 222)
    x.random_(0, 256, generator=g)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    for kb in (128, 256):
        enc, dec, nr = aesgb.aes_expand_key(kb, wl.random_key(kb, 222).tobytes())
        aesgb.aes_ecb_encrypt(enc, nr, x, y1, n)
        aesgb.aes_ecb_crypt_ct(0, enc, nr, x, y2, n)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        aesgb.aes_ecb_decrypt(dec, nr, y1, y1, n)
        aesgb.aes_ecb_crypt_ct(1, dec, nr, y2, y2, n)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2) and torch.equal(y1, x)


def test_logic_rate_calibration():
    """The LOP3 calibration kernel measures a rate in the range the hardware
    allows: positive, and at most 64 lanes per clock per SM at the highest
    SM clock the device reports (a rate above it would mean the kernel did
    not do the work it counts)."""
    torch = torch_cuda()
    sms = aesgb.aes_device_sm_count(0)
    sink = torch.empty(sms * 4096, dtype=torch.uint8, device="cuda")
    ops, secs = aesgb.aes_calibrate_logic_rate(sink, sink.numel())
    assert ops > 0 and secs > 0
    clock_hz = torch.cuda.get_device_properties(0).clock_rate * 1e3 if hasattr(
        torch.cuda.get_device_properties(0), "clock_rate") else 2.1e9
    per_sm_per_clk = ops / secs / (sms * clock_hz)
    assert 16 < per_sm_per_clk <= 64 * 1.05, per_sm_per_clk
    with pytest.raises(aesgb.AesError):
        aesgb.aes_calibrate_logic_rate(sink, 16)
