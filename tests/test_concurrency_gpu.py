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
