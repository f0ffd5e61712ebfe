"""The entry points are capturable in a CUDA graph (they neither allocate nor
synchronise once warmed up) and safe to call from several host threads on
distinct streams at once; results stay bit-exact."""
import threading

import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from batch_util import DeviceBatch
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_single_buffer_calls_in_a_cuda_graph(orc):
    torch = torch_cuda()
    key = wl.random_key(192, 230).tobytes()
    enc, dec, nr = aesgb.aes_expand_key(192, key)
    n = 50_001
    data = wl.random_bytes(16 * n, 230)
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):                       # warm-up: attributes, occupancy, tuning cache
        aesgb.aes_ecb_encrypt(enc, nr, x, y, n, s)
        aesgb.aes_ecb_decrypt(dec, nr, y, z, n, s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        aesgb.aes_ecb_encrypt(enc, nr, x, y, n, s)
        aesgb.aes_ecb_decrypt(dec, nr, y, z, n, s)
    y.zero_()
    z.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), orc.ecb(0, key, data, nthreads=8))
    assert torch.equal(z, x)


def test_concurrent_host_threads_on_distinct_streams(orc):
    torch = torch_cuda()
    errors = []
    results = {}

    def worker(tid):
        try:
            s = torch.cuda.Stream()
            kb = (128, 192, 256, 128)[tid]
            key = wl.random_key(kb, 240 + tid).tobytes()
            enc, dec, nr = aesgb.aes_expand_key(kb, key)
            n = 100_000 + 1000 * tid
            data = wl.random_bytes(16 * n, 240 + tid)
            with torch.cuda.stream(s):
                x = torch.from_numpy(data).cuda()
                y = torch.empty_like(x)
                z = torch.empty_like(x)
                for _ in range(20):
                    aesgb.aes_ecb_encrypt(enc, nr, x, y, n, s)
                    aesgb.aes_ecb_decrypt(dec, nr, y, z, n, s)
                    aesgb.aes_ctr_crypt(enc, nr, bytes(16), z, z, n, s)
                    aesgb.aes_ctr_crypt(enc, nr, bytes(16), z, z, n, s)
                b = DeviceBatch(torch, [16 * 7, 4096, 65536], [kb] * 3, [0, 1, 0], seed=250 + tid)
                ws, nbytes = b.workspace()
                aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, stream=s)
            s.synchronize()
            results[tid] = (key, data, y.cpu().numpy(), bool(torch.equal(z, x)), b, b.output())
        except Exception as e:  # pragma: no cover - reported below
            errors.append((tid, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for tid, (key, data, ct, roundtrip, b, bout) in results.items():
        assert roundtrip, tid
        assert np.array_equal(ct, orc.ecb(0, key, data, nthreads=8)), tid
        for i in range(b.n):
            exp = orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i))
            assert np.array_equal(b.message(bout, i), exp), (tid, i)


def _pooled_batch(torch, n, hi, seed, pool=6):
    """n messages of 16..hi bytes (log-uniform), each under one of `pool`
    random keys of mixed size and a random direction, packed back to back.
    Returns the device tensors and, per (key, direction) group, the message
    slices, so that the oracle can take each group's messages in one ECB call
    (ECB is blockwise, so concatenating messages of one key concatenates their
    outputs)."""
    g = wl.rng(seed)
    lengths = wl.log_uniform_lengths(n, 16, hi, g)
    kbits = [int(k) for k in g.choice(np.array([128, 192, 256]), size=pool)]
    keys = [wl.random_key(kb, seed * 10 + j).tobytes() for j, kb in enumerate(kbits)]
    kid = g.integers(0, pool, size=n)
    dirs = g.integers(0, 2, size=n)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=offs[1:])
    data = wl.random_bytes(int(offs[-1]), seed)
    rks = np.zeros((2 * pool, 64), np.uint32)                 # row 2j + dir: key j's schedule
    nrs = np.zeros(pool, np.int64)
    for j in range(pool):
        e, d, nrs[j] = aesgb.aes_expand_key(kbits[j], keys[j])
        rks[2 * j, :60], rks[2 * j + 1, :60] = e, d
    x = torch.from_numpy(data).cuda()
    y = torch.full_like(x, 0x5A)
    rk = torch.from_numpy(rks.view(np.uint8).reshape(-1)).cuda()
    table = aesgb.pack_descs(rk.data_ptr() + 256 * (2 * kid + dirs).astype(np.uint64),
                             x.data_ptr() + offs[:-1].astype(np.uint64),
                             y.data_ptr() + offs[:-1].astype(np.uint64),
                             lengths // 16, nrs[kid], dirs)
    desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
    groups = {}
    for i in range(n):
        groups.setdefault((int(kid[i]), int(dirs[i])), []).append(slice(int(offs[i]), int(offs[i + 1])))
    return dict(x=x, y=y, rk=rk, desc=desc, n=n, data=data, keys=keys, groups=groups)


def _check_pooled(orc, b, out):
    for (j, d), parts in b["groups"].items():
        src = np.concatenate([b["data"][p] for p in parts])
        got = np.concatenate([out[p] for p in parts])
        assert np.array_equal(got, orc.ecb(d, b["keys"][j], src, nthreads=4)), (j, d)


def test_library_workspace_batches_from_four_threads_at_once(orc):
    """aes_ecb_batch from four host threads at once, each on its own stream,
    each with three batches of different sizes queued back to back: the third
    (about 56,000 descriptors, above the 1 MiB first workspace) makes every
    stream's workspace grow while the first two batches may still be queued.
    Each output equals the oracle bit for bit.  A long run of launches on a
    fifth stream is still executing when every call has returned, which shows
    that no call (growth included) waited for the device."""
    torch = torch_cuda()
    aesgb.aes_shutdown()                                   # every stream starts without a workspace
    sizes = [200, 5_000, 56_000]
    batches = {t: [_pooled_batch(torch, sizes[k] + 500 * t, (1 << 12) if k < 2 else 64, 700 + 10 * t + k)
                   for k in range(3)] for t in range(4)}
    streams = {t: torch.cuda.Stream() for t in range(4)}
    # the blocker: 1 GiB encrypted in place 128 times (well over 100 ms)
    blk = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    enc, _, nr = aesgb.aes_expand_key(128, bytes(16))
    bs = torch.cuda.Stream()
    aesgb.aes_ecb_encrypt(enc, nr, blk, blk, blk.numel() // 16, bs)   # warm-up (attributes, occupancy)
    for t in range(4):                                     # warm-up of the batch kernel set-up, 1 descriptor
        aesgb.aes_ecb_batch(batches[t][0]["desc"], 1, streams[t])
    torch.cuda.synchronize()
    for t in range(4):
        batches[t][0]["y"].fill_(0x5A)
    aesgb.aes_shutdown()
    torch.cuda.synchronize()
    blocker_done = torch.cuda.Event()
    for _ in range(128):
        aesgb.aes_ecb_encrypt(enc, nr, blk, blk, blk.numel() // 16, bs)
    blocker_done.record(bs)

    errors = []
    go = threading.Barrier(4)

    def worker(t):
        try:
            go.wait(timeout=30)
            for b in batches[t]:
                aesgb.aes_ecb_batch(b["desc"], b["n"], streams[t])
        except Exception as e:  # pragma: no cover - reported below
            errors.append((t, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    still_running = not blocker_done.query()
    torch.cuda.synchronize()
    assert not errors, errors
    assert still_running, "an aes_ecb_batch call waited for work on another stream"
    for t in range(4):
        for b in batches[t]:
            _check_pooled(orc, b, b["y"].cpu().numpy())


def test_library_workspace_batch_refuses_a_capturing_stream(orc):
    """aes_ecb_batch on a stream under graph capture answers AES_E_CONFIG and
    enqueues nothing; aes_ecb_batch_ws with a caller-owned workspace is the
    capturable form, and its replay is exact."""
    torch = torch_cuda()
    b = _pooled_batch(torch, 300, 1 << 12, 790)
    ws = torch.empty(max(aesgb.aes_batch_workspace_bytes(b["n"]), 256), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    aesgb.aes_ecb_batch_ws(b["desc"], b["n"], ws, ws.numel(), stream=s)   # set-up before capture
    s.synchronize()
    b["y"].fill_(0x5A)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_ecb_batch(b["desc"], b["n"], s)
        aesgb.aes_ecb_batch_ws(b["desc"], b["n"], ws, ws.numel(), stream=s)
    assert e.value.status == -12
    torch.cuda.synchronize()
    assert bool((b["y"] == 0x5A).all())                 # nothing ran at capture time
    g.replay()
    torch.cuda.synchronize()
    _check_pooled(orc, b, b["y"].cpu().numpy())


def test_library_workspaces_of_many_streams(orc):
    """More than 64 streams each run a batch through the library workspace:
    once 64 per-stream workspaces exist, the idle ones of other streams are
    released as new streams arrive.  Every stream's output stays exact, and
    reusing an early stream (its workspace released) allocates a new one."""
    torch = torch_cuda()
    aesgb.aes_shutdown()
    b = _pooled_batch(torch, 40, 1 << 10, 795)
    streams = [torch.cuda.Stream() for _ in range(80)]
    for s in streams:
        b["y"].fill_(0x5A)
        torch.cuda.synchronize()
        aesgb.aes_ecb_batch(b["desc"], b["n"], s)
        s.synchronize()
        _check_pooled(orc, b, b["y"].cpu().numpy())
    b["y"].fill_(0x5A)
    torch.cuda.synchronize()
    aesgb.aes_ecb_batch(b["desc"], b["n"], streams[0])
    streams[0].synchronize()
    _check_pooled(orc, b, b["y"].cpu().numpy())
    aesgb.aes_shutdown()
