"""aes_ecb_batch_noalloc: the batched entry point for callers that must not
allocate device memory (plugins that may only touch the buffers their host
hands them, code running during another thread's global-mode graph capture,
serving threads that cannot let cudaMalloc/cudaFree synchronise the device).
Its workspace is a fixed array inside the library, so this test checks, through
the C ABI, that two calls in a row -- a larger batch, then a smaller one that
reuses the array the first one left behind, with a host synchronisation
between them or queued back to back on one stream -- give exactly what the
workspace-taking entry point aes_ecb_batch_ws gives and what the oracle gives
(integer work: bit-exact), and that a batch above the documented maximum is refused before anything is
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


def _check_against_oracle(orc, b: DeviceBatch, out, skip=()):
    """Every message of up to 64 KiB whole, and the first and last 2 KiB of
    each larger one (ECB is blockwise), against the oracle; messages in
    `skip` (invalid descriptors) must be untouched."""
    for i in range(b.n):
        got = b.message(out, i)
        if i in skip:
            assert np.all(got == 0x5A), i
            continue
        src = b.message(b.data, i)
        d, key = int(b.dirs[i]), b.keys[i]
        if src.size <= 64 * 1024:
            assert np.array_equal(got, orc.ecb(d, key, src)), i
        else:
            for w in (slice(0, 2048), slice(src.size - 2048, src.size)):
                assert np.array_equal(got[w], orc.ecb(d, key, src[w])), (i, w)


def test_no_alloc_batch_matches_workspace_batch_twice(orc):
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
    _check_against_oracle(orc, first, got1, skip=(3,))
    _check_against_oracle(orc, second, got2)


def test_no_alloc_batches_queued_back_to_back_on_one_stream(orc):
    """The documented safe pattern: two calls queued on one stream with no
    synchronisation between them, so the second call's plan kernel rewrites
    the shared scratch right behind the first call's batch kernel.  Stream
    order keeps them apart: outputs and statuses equal those of
    aes_ecb_batch_ws, and the oracle's."""
    torch = torch_cuda()
    first = DeviceBatch(torch, *_mix(500, 63, 1 << 20), seed=63)
    first.table[7]["dir"] = 2               # one invalid descriptor: skipped, status set
    first.upload()
    second = DeviceBatch(torch, *_mix(300, 64, 1 << 18), seed=64)
    exp1, st1 = _reference(torch, first)
    exp2, st2 = _reference(torch, second)
    s = torch.cuda.Stream()
    status1 = torch.full((first.n,), 77, dtype=torch.int32, device="cuda")
    status2 = torch.full((second.n,), 77, dtype=torch.int32, device="cuda")
    first.out_dev.fill_(0x5A)
    second.out_dev.fill_(0x5A)
    torch.cuda.synchronize()
    aesgb.aes_ecb_batch_noalloc(first.desc_dev, first.n, status1, s)
    aesgb.aes_ecb_batch_noalloc(second.desc_dev, second.n, status2, s)
    s.synchronize()
    got1, got2 = first.output().copy(), second.output().copy()
    assert np.array_equal(got1, exp1) and np.array_equal(got2, exp2)
    assert np.array_equal(status1.cpu().numpy(), st1) and st1[7] == -1
    assert np.array_equal(status2.cpu().numpy(), st2) and np.all(st2 == 0)
    _check_against_oracle(orc, first, got1, skip=(7,))
    _check_against_oracle(orc, second, got2)


def test_no_alloc_batch_rejects_oversized_batch():
    torch_cuda()
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_ecb_batch_noalloc(0, aesgb.AES_BATCH_NOALLOC_MAX_DESCS + 1)
    assert e.value.status == -10                 # AES_E_RANGE, nothing queued
    aesgb.aes_ecb_batch_noalloc(0, 0)            # an empty batch is a no-op
