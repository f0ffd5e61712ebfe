"""CTR (eq (5)) and CBC decryption (eq (2), parallel form) on the GPU,
bit-exact against the oracle (itself pinned to OpenSSL), and ECB directly on
page-locked host memory."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 32, 33, 1025, 4097, 100_003]


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_ctr_matches_oracle(orc, keybits):
    torch = torch_cuda()
    key = wl.random_key(keybits, 90).tobytes()
    enc, _, nr = aesgb.aes_expand_key(keybits, key)
    g = wl.rng(90 + keybits)
    for n in SIZES:
        data = wl.random_bytes(16 * n, 91 + n)
        ctr0 = g.integers(0, 256, 16, dtype=np.uint8)
        x = torch.from_numpy(data).cuda()
        y = torch.full_like(x, 0x5A)
        aesgb.aes_ctr_crypt(enc, nr, ctr0, x, y, n)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), orc.ctr(key, ctr0, data)), n
        aesgb.aes_ctr_crypt(enc, nr, ctr0, y, y, n)          # the same call decrypts, in place
        torch.cuda.synchronize()
        assert torch.equal(y, x)


def test_ctr_counter_wraps(orc):
    torch = torch_cuda()
    key = wl.random_key(128, 92).tobytes()
    enc, _, nr = aesgb.aes_expand_key(128, key)
    n = 5000
    data = wl.random_bytes(16 * n, 92)
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    wrap64 = np.zeros(16, np.uint8)
    wrap64[8:] = 0xFF
    wrap64[15] = 0x00                                     # low half = 2^64 - 256: wraps inside the buffer
    wrap128 = np.full(16, 0xFF, np.uint8)
    wrap128[14:] = [0xF0, 0x00]                           # 2^128 - 4096: wraps to zero inside the buffer
    for ctr0 in (wrap64, wrap128):
        aesgb.aes_ctr_crypt(enc, nr, ctr0, x, y, n)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), orc.ctr(key, ctr0, data))


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_cbc_decrypt_matches_oracle(orc, keybits):
    torch = torch_cuda()
    key = wl.random_key(keybits, 93).tobytes()
    _, dec, nr = aesgb.aes_expand_key(keybits, key)
    g = wl.rng(93 + keybits)
    for n in SIZES + [200_003]:                           # the last spans several grid passes
        iv = g.integers(0, 256, 16, dtype=np.uint8)
        ct = wl.random_bytes(16 * n, 94 + n)
        x = torch.from_numpy(ct).cuda()
        y = torch.full_like(x, 0x5A)
        aesgb.aes_cbc_decrypt(dec, nr, iv, x, y, n)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), orc.cbc_decrypt(key, iv, ct)), n
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_cbc_decrypt(dec, nr, iv, x, x, 16)
    assert e.value.status == -5


def test_cbc_roundtrip_with_oracle_encryption(orc):
    """Ciphertext made by the oracle's (sequential) CBC encryption decrypts back."""
    torch = torch_cuda()
    key = wl.random_key(256, 95).tobytes()
    _, dec, nr = aesgb.aes_expand_key(256, key)
    iv = wl.random_bytes(16, 95)
    pt = wl.random_bytes(16 * 70_001, 96)
    ct = orc.cbc_encrypt(key, iv, pt)
    x = torch.from_numpy(ct).cuda()
    y = torch.empty_like(x)
    aesgb.aes_cbc_decrypt(dec, nr, iv, x, y, pt.size // 16)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), pt)


def test_ecb_host_direct(orc):
    torch = torch_cuda()
    key = wl.random_key(192, 97).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(192, key)
    n = 123_457
    data = wl.random_bytes(16 * n, 97)
    h_in = torch.from_numpy(data.copy()).pin_memory()
    h_out = torch.zeros_like(h_in).pin_memory()
    s = torch.cuda.current_stream()
    aesgb.aes_ecb_host_direct(0, enc, nr, h_in, h_out, n, s)
    s.synchronize()
    assert np.array_equal(h_out.numpy(), orc.ecb(0, key, data, nthreads=8))
    aesgb.aes_ecb_host_direct(1, dec, nr, h_out, h_out, n, s)      # in place
    s.synchronize()
    assert np.array_equal(h_out.numpy(), data)
    pageable = torch.from_numpy(data.copy())
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_ecb_host_direct(0, enc, nr, pageable, h_out, n, s)
    assert e.value.status == -1


@pytest.mark.parametrize("keybits", [128, 192, 256])
def test_cfb_decrypt_matches_oracle(orc, keybits):
    """CFB decryption (full-block CFB; the forward cipher on the previous
    ciphertext block) against the oracle, ragged sizes and several grid
    passes; in place is refused."""
    torch = torch_cuda()
    key = wl.random_key(keybits, 97).tobytes()
    enc, _, nr = aesgb.aes_expand_key(keybits, key)
    g = wl.rng(97 + keybits)
    for n in SIZES + [200_003]:
        iv = g.integers(0, 256, 16, dtype=np.uint8)
        ct = wl.random_bytes(16 * n, 98 + n)
        x = torch.from_numpy(ct).cuda()
        y = torch.full_like(x, 0x5A)
        aesgb.aes_cfb_decrypt(enc, nr, iv, x, y, n)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), orc.cfb_decrypt(key, iv, ct)), n
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_cfb_decrypt(enc, nr, iv, x, x, 16)
    assert e.value.status == -5


def test_cfb_roundtrip_with_oracle_encryption(orc):
    """Ciphertext made by the oracle's (sequential) CFB encryption decrypts back."""
    torch = torch_cuda()
    key = wl.random_key(192, 99).tobytes()
    enc, _, nr = aesgb.aes_expand_key(192, key)
    iv = wl.random_bytes(16, 99)
    pt = wl.random_bytes(16 * 70_001, 100)
    ct = orc.cfb_encrypt(key, iv, pt)
    x = torch.from_numpy(ct).cuda()
    y = torch.empty_like(x)
    aesgb.aes_cfb_decrypt(enc, nr, iv, x, y, pt.size // 16)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), pt)
