"""Continuous-batching server: every result bit-exact against the oracle,
identical alone and in the mix; admission within the device-memory budget;
open-loop (arrival-time) submission; bounded waits; argument errors."""
import numpy as np
import pytest

from paper_1902_05234_gb300 import aesgb
from paper_1902_05234_gb300 import workloads as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


class Arena:
    """Requests' input and output buffers packed in two device arenas."""

    def __init__(self, torch, sizes, seed):
        self.sizes = np.asarray(sizes, np.int64)
        self.offs = np.zeros(len(sizes) + 1, np.int64)
        np.cumsum(self.sizes, out=self.offs[1:])
        total = int(self.offs[-1])
        self.data = wl.random_bytes(total, seed)
        self.inp = torch.from_numpy(self.data).cuda()
        self.out = torch.full((total,), 0x5A, dtype=torch.uint8, device="cuda")

    def ins(self):
        return self.inp.data_ptr() + self.offs[:-1].astype(np.uint64)

    def outs(self, buf=None):
        return (buf if buf is not None else self.out).data_ptr() + self.offs[:-1].astype(np.uint64)

    def msg(self, arr, i):
        return arr[self.offs[i]:self.offs[i + 1]]


@pytest.fixture()
def server():
    torch_cuda()
    srv = aesgb.aes_srv_create(64 << 20, max_keys=32, max_batch=256, slots=3)
    keys = {}
    g = wl.rng(70)
    for k in range(32):
        kb = (128, 192, 256)[k % 3]
        keys[k] = (kb, g.integers(0, 256, kb // 8, dtype=np.uint8).tobytes())
        aesgb.aes_srv_put_key(srv, k, kb, keys[k][1])
    yield srv, keys
    aesgb.aes_srv_destroy(srv)


def test_served_mix_matches_oracle_and_alone(orc, server):
    torch = torch_cuda()
    srv, keys = server
    n = 600
    arrivals, sizes, key_ids, dirs = wl.served_workload(n, rate_per_s=20000.0, n_keys=32, hi=256 * 1024,
                                                        seed_offset=71)
    a = Arena(torch, sizes, 72)
    st, tickets = aesgb.aes_srv_submit_many(srv, key_ids, dirs, a.ins(), a.outs(), sizes,
                                            arrivals - arrivals[0])
    assert st == 0 and np.all(tickets > 0)
    aesgb.aes_srv_drain(srv, 60000)
    status, lat, queue = aesgb.aes_srv_results(srv, tickets)
    assert np.all(status == 0)
    assert np.all(lat > 0) and np.all(queue >= 0)
    out = a.out.cpu().numpy()
    for i in range(n):
        kb, key = keys[int(key_ids[i])]
        exp = orc.ecb(int(dirs[i]), key, a.msg(a.data, i), nthreads=1)
        assert np.array_equal(a.msg(out, i), exp), i
    stats = aesgb.aes_srv_stats(srv)
    assert stats["completed"] == n and stats["batches"] >= 1 and stats["worker_status"] == 0
    # alone: a sample of the same requests, one at a time, into fresh buffers
    alone = torch.full_like(a.out, 0x33)
    outs_alone = a.outs(alone)
    for i in range(0, n, 29):
        t = aesgb.aes_srv_submit(srv, int(key_ids[i]), int(dirs[i]), int(a.ins()[i]), int(outs_alone[i]),
                                 int(sizes[i]))
        s, _ = aesgb.aes_srv_wait(srv, t, 10000)
        assert s == 0
    alone_h = alone.cpu().numpy()
    for i in range(0, n, 29):
        assert np.array_equal(a.msg(alone_h, i), a.msg(out, i)), i


def test_budget_caps_bytes_in_flight(orc, server):
    torch = torch_cuda()
    srv0, keys = server
    budget = 4 << 20                                       # 4 MiB: at most 2 MiB of requests in flight
    srv = aesgb.aes_srv_create(budget, max_keys=4, max_batch=64, slots=4)
    try:
        for k in range(4):
            aesgb.aes_srv_put_key(srv, k, keys[k][0], keys[k][1])
        sizes = np.full(200, 256 * 1024, np.int64)
        a = Arena(torch, sizes, 73)
        kid = np.arange(200) % 4
        dirs = np.arange(200) % 2
        st, tickets = aesgb.aes_srv_submit_many(srv, kid, dirs, a.ins(), a.outs(), sizes)
        assert st == 0
        aesgb.aes_srv_drain(srv, 60000)
        stats = aesgb.aes_srv_stats(srv)
        assert stats["completed"] == 200
        assert 0 < stats["peak_inflight_bytes"] <= budget
        assert stats["batches"] >= 200 * 2 * 256 * 1024 // budget
        out = a.out.cpu().numpy()
        for i in range(0, 200, 13):
            exp = orc.ecb(int(dirs[i]), keys[int(kid[i])][1], a.msg(a.data, i), nthreads=4)
            assert np.array_equal(a.msg(out, i), exp)
        # a request that can never fit the budget is refused at submission
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_submit(srv, 0, 0, a.inp, a.out, budget)
        assert e.value.status == -10
    finally:
        aesgb.aes_srv_destroy(srv)


def test_errors_and_bounded_wait(server):
    torch = torch_cuda()
    srv, _ = server
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(aesgb.AesError) as e:
        aesgb.aes_srv_submit(srv, 99, 0, buf, buf, 4096)        # key id out of range
    assert e.value.status == -11
    srv2 = aesgb.aes_srv_create(1 << 20, max_keys=2, max_batch=8, slots=1)
    try:
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_submit(srv2, 1, 0, buf, buf, 4096)   # key never put
        assert e.value.status == -11
        aesgb.aes_srv_put_key(srv2, 0, 128, bytes(16))
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_submit(srv2, 0, 0, buf, buf, 4008)   # not a multiple of 16
        assert e.value.status == -1
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_submit(srv2, 0, 0, buf.data_ptr() + 8, buf, 16)
        assert e.value.status == -4
        # a request that arrives 30 s from now: a short wait times out on the host
        st, t = aesgb.aes_srv_submit_many(srv2, [0], [0], [buf.data_ptr()], [buf.data_ptr()], [4096], [30.0])
        assert st == 0
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_wait(srv2, int(t[0]), 50)
        assert e.value.status == -8
        done, _, _ = aesgb.aes_srv_poll(srv2, int(t[0]))
        assert not done
    finally:
        aesgb.aes_srv_destroy(srv2)                             # drops the future request
