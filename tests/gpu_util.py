"""Helpers for the GPU parity tests: move seeded inputs to the device, call
the C ABI, bring results back.  Expected values always come from the oracle."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(torch, arr: np.ndarray, pad_front: int = 0, pad_back: int = 0, fill: int = 0xA5):
    """Copy host bytes into a fresh device buffer with optional guard bytes."""
    buf = torch.full((pad_front + arr.size + pad_back,), fill, dtype=torch.uint8, device="cuda")
    if arr.size:
        buf[pad_front:pad_front + arr.size].copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    return buf


def gpu_ecb(direction, key, data: np.ndarray, cfg=None, inplace=False, guard=0):
    """Run one ECB call through the C ABI on `data`; returns (result, guards_ok)."""
    torch = torch_cuda()
    kb = 8 * len(key)
    enc, dec, nr = aesgb.aes_expand_key(kb, key)
    rk = enc if direction == 0 else dec
    n = data.size // 16
    src = to_dev(torch, data, guard, guard)
    if inplace:
        dst = src
    else:
        dst = torch.full((guard + data.size + guard,), 0x5A, dtype=torch.uint8, device="cuda")
    ip = src.data_ptr() + guard
    op = dst.data_ptr() + guard
    if cfg is None:
        (aesgb.aes_ecb_encrypt if direction == 0 else aesgb.aes_ecb_decrypt)(rk, nr, ip, op, n)
    else:
        aesgb.aes_ecb_crypt_cfg(direction, rk, nr, ip, op, n, cfg)
    torch.cuda.synchronize()
    host = dst.cpu().numpy()
    out = host[guard:guard + data.size].copy()
    ok = True
    if guard:
        fill = 0xA5 if inplace else 0x5A
        ok = bool(np.all(host[:guard] == fill) and np.all(host[guard + data.size:] == fill))
    return out, ok
