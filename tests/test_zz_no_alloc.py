"""aes_ecb_batch_noalloc: the batched entry point for callers that must not
allocate device memory (plugins that may only touch the buffers their host
hands them, code running during another thread's global-mode graph capture,
serving threads that cannot let cudaMalloc/cudaFree synchronise the device).
Its workspace is a fixed array inside the library, so this test checks, through
the C ABI, that two calls in a row -- a larger batch, then a smaller one that
reuses the array the first one left behind -- give exactly what the
workspace-taking entry point aes_ecb_batch_ws gives (integer work: bit-exact),
and that a batch above the documented maximum is refused before anything is
queued.  It runs last (file name) and needs nothing from the other tests."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from batch_util import DeviceBatch
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _mix(n, seed, hi):
    g = wl.rng(seed)
    lengths = wl.log_uniform_lengths(n, 16, hi, g)
    keybits = g.choice(np.array([128, 192, 256]), size=n)
    dirs = g.integers(0, 2, size=n)
    return lengths, keybits, dirs


def _reference(torch, b: DeviceBatch):
    """Output and statuses of the same batch through aes_ecb_batch_ws."""
    ws, nbytes = b.workspace()
    status = torch.full((b.n,), 77, dtype=torch.int32, device="cuda")
    b.out_dev.fill_(0x5A)
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, status)
    out = b.output().copy()
    return out, status.cpu().numpy()


def _no_alloc(torch, b: DeviceBatch):
    status = torch.full((b.n,), 77, dtype=torch.int32, device="cuda")
    b.out_dev.fill_(0x5A)
    aesgb.aes_ecb_batch_noalloc(b.desc_dev, b.n, status)
    return b.output().copy(), status.cpu().numpy()


def test_no_alloc_batch_matches_workspace_batch_twice():
    torch = torch_cuda()
    first = DeviceBatch(torch, *_mix(700, 61, 1 << 20), seed=61)
    first.table[3]["nrounds"] = 13          # one invalid descriptor: skipped, status set
    first.upload()
    second = DeviceBatch(torch, *_mix(90, 62, 1 << 16), seed=62)

    exp1, st1 = _reference(torch, first)
    exp2, st2 = _reference(torch, second)

    got1, gst1 = _no_alloc(torch, first)    # call 1
    got2, gst2 = _no_alloc(torch, second)   # call 2, right after, same scratch array
    assert np.array_equal(got1, exp1)
    assert np.array_equal(gst1, st1) and gst1[3] == -3
    assert np.array_equal(got2, exp2)
    assert np.array_equal(gst2, st2) and np.all(gst2 == 0)


def test_no_alloc_batch_rejects_oversized_batch():
    torch_cuda()
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_ecb_batch_noalloc(0, aesgb.AES_BATCH_NOALLOC_MAX_DESCS + 1)
    assert e.value.status == -10                 # AES_E_RANGE, nothing queued
    aesgb.aes_ecb_batch_noalloc(0, 0)            # an empty batch is a no-op
