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


def _check_windows(orc, key, dirn, src, got, whole=64 * 1024, win=2048):
    """A served result against the oracle: whole up to `whole` bytes, else its
    first and last `win` bytes (ECB is blockwise)."""
    if src.size <= whole:
        return np.array_equal(got, orc.ecb(dirn, key, src, nthreads=1))
    return all(np.array_equal(got[w], orc.ecb(dirn, key, src[w], nthreads=1))
               for w in (slice(0, win), slice(src.size - win, src.size)))


def test_served_workload_ranges_match_oracle_and_alone(orc):
    """The served workload's ranges: request sizes log-uniform from 64 B to
    4 MiB, 1,024 resident keys of mixed size, Poisson arrivals, a 4 GiB
    budget over 4 slots.  Every result against the oracle (whole up to
    64 KiB, the first and last 2 KiB above), and a sample re-run alone into
    fresh buffers is identical to its result in the mix."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(4 << 30, max_keys=1024, max_batch=4096, slots=4)
    try:
        g = wl.rng(75)
        keys = {}
        for k in range(1024):
            kb = int(g.choice(np.array([128, 192, 256])))
            keys[k] = g.integers(0, 256, kb // 8, dtype=np.uint8).tobytes()
            aesgb.aes_srv_put_key(srv, k, kb, keys[k])
        n = 800
        arrivals, sizes, key_ids, dirs = wl.served_workload(n, rate_per_s=20000.0, n_keys=1024, seed_offset=76)
        assert sizes.min() >= 64 and sizes.max() <= 4 << 20 and sizes.max() > 1 << 20
        a = Arena(torch, sizes, 77)
        st, tickets = aesgb.aes_srv_submit_many(srv, key_ids, dirs, a.ins(), a.outs(), sizes,
                                                arrivals - arrivals[0])
        assert st == 0 and np.all(tickets > 0)
        aesgb.aes_srv_drain(srv, 120000)
        status, lat, _ = aesgb.aes_srv_results(srv, tickets)
        assert np.all(status == 0) and np.all(lat > 0)
        out = a.out.cpu().numpy()
        for i in range(n):
            key = keys[int(key_ids[i])]
            assert _check_windows(orc, key, int(dirs[i]), a.msg(a.data, i), a.msg(out, i)), i
        stats = aesgb.aes_srv_stats(srv)
        assert stats["completed"] == n and stats["worker_status"] == 0
        assert 0 < stats["peak_inflight_bytes"] <= 4 << 30
        alone = torch.full_like(a.out, 0x33)
        outs_alone = a.outs(alone)
        sample = list(range(0, n, 37)) + [int(np.argmax(sizes))]
        for i in sample:
            t = aesgb.aes_srv_submit(srv, int(key_ids[i]), int(dirs[i]), int(a.ins()[i]), int(outs_alone[i]),
                                     int(sizes[i]))
            s_, _ = aesgb.aes_srv_wait(srv, t, 10000)
            assert s_ == 0
        alone_h = alone.cpu().numpy()
        for i in sample:
            assert np.array_equal(a.msg(alone_h, i), a.msg(out, i)), i
    finally:
        aesgb.aes_srv_destroy(srv)


def test_batches_overlap_on_the_device(orc):
    """Continuous batching: a 1 GiB AES-256 request takes one slot, and small
    requests that arrive while it runs are packed into batches on the other
    slots.  The stats show two or more slots busy at once and, from the
    batches' device intervals, a later batch's stream reaching its kernel
    before the long batch's kernel completed.  Every result equals the oracle
    (the long one in windows) and its re-run alone."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(4 << 30, max_keys=4, max_batch=1024, slots=4)
    try:
        keys = {k: wl.random_key((256, 128, 192, 256)[k], 410 + k).tobytes() for k in range(4)}
        for k in range(4):
            aesgb.aes_srv_put_key(srv, k, 8 * len(keys[k]), keys[k])
        aesgb.aes_srv_set_device_timing(srv, True)
        big_n = 1 << 30
        gen = torch.Generator(device="cuda").manual_seed(190205230 + 411)
        big_in = torch.randint(0, 256, (big_n,), dtype=torch.uint8, device="cuda", generator=gen)
        big_out = torch.full_like(big_in, 0x5A)
        m = 240
        g = wl.rng(412)
        sizes = wl.log_uniform_lengths(m, 64, 64 * 1024, g)
        kid = g.integers(0, 4, size=m)
        dirs = g.integers(0, 2, size=m)
        a = Arena(torch, sizes, 413)
        offsets = np.concatenate([[0.0], np.linspace(1e-4, 2e-3, m)])   # small ones over 2 ms
        ins = np.concatenate([[big_in.data_ptr()], a.ins()]).astype(np.uint64)
        outs = np.concatenate([[big_out.data_ptr()], a.outs()]).astype(np.uint64)
        st, tickets = aesgb.aes_srv_submit_many(srv, np.concatenate([[0], kid]), np.concatenate([[1], dirs]),
                                                ins, outs, np.concatenate([[big_n], sizes]), offsets)
        assert st == 0 and np.all(tickets > 0)
        aesgb.aes_srv_drain(srv, 60000)
        status, _, _ = aesgb.aes_srv_results(srv, tickets)
        assert np.all(status == 0)
        stats = aesgb.aes_srv_stats(srv)
        assert stats["batches"] >= 3 and stats["timed_batches"] == stats["batches"]
        assert stats["peak_busy_slots"] >= 2, stats
        assert stats["peak_device_batches"] >= 2 and stats["device_overlap_s"] > 0, stats
        out = a.out.cpu().numpy()
        for i in range(m):
            assert _check_windows(orc, keys[int(kid[i])], int(dirs[i]), a.msg(a.data, i), a.msg(out, i)), i
        for off in (0, big_n // 2 - 4096, big_n - 65536):
            w = slice(off, off + 65536)
            src = big_in[w].cpu().numpy()
            assert np.array_equal(big_out[w].cpu().numpy(), orc.ecb(1, keys[0], src, nthreads=4)), off
        # alone: the long request and every 9th small one, into fresh buffers
        big_alone = torch.full_like(big_in, 0x33)
        t = aesgb.aes_srv_submit(srv, 0, 1, big_in, big_alone, big_n)
        s_, _ = aesgb.aes_srv_wait(srv, t, 20000)
        assert s_ == 0 and torch.equal(big_alone, big_out)
        alone = torch.full_like(a.out, 0x33)
        for i in range(0, m, 9):
            t = aesgb.aes_srv_submit(srv, int(kid[i]), int(dirs[i]), int(a.ins()[i]), int(a.outs(alone)[i]),
                                     int(sizes[i]))
            s_, _ = aesgb.aes_srv_wait(srv, t, 10000)
            assert s_ == 0
        alone_h = alone.cpu().numpy()
        for i in range(0, m, 9):
            assert np.array_equal(a.msg(alone_h, i), a.msg(out, i)), i
    finally:
        aesgb.aes_srv_destroy(srv)


def test_device_timing_is_off_by_default():
    """Without aes_srv_set_device_timing no batch carries timing events (no
    device intervals), while the host-side counters are kept; switched on, the
    next busy period's batches are timed."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(8 << 20, max_keys=1, max_batch=16, slots=2)
    try:
        aesgb.aes_srv_put_key(srv, 0, 128, bytes(16))
        x = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            aesgb.aes_srv_wait(srv, aesgb.aes_srv_submit(srv, 0, 0, x, y, x.numel()), 10000)
        st = aesgb.aes_srv_stats(srv)
        assert st["batches"] == 3 and st["timed_batches"] == 0 and st["peak_busy_slots"] >= 1
        assert st["peak_device_batches"] == 0 and st["device_overlap_s"] == 0.0
        aesgb.aes_srv_set_device_timing(srv, True)
        for _ in range(2):
            aesgb.aes_srv_wait(srv, aesgb.aes_srv_submit(srv, 0, 0, x, y, x.numel()), 10000)
        st = aesgb.aes_srv_stats(srv)
        assert st["batches"] == 5 and st["timed_batches"] == 2 and st["peak_device_batches"] >= 1
    finally:
        aesgb.aes_srv_destroy(srv)


def test_put_key_refused_while_a_request_names_it(orc):
    """A queued request keeps its key: replacing the key it names answers
    AES_E_BUSY until the request is gone (here: cancelled).  The replacement,
    of another size, is then used by the next request, and other keys can be
    replaced meanwhile."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(8 << 20, max_keys=2, max_batch=16, slots=2)
    try:
        k128, k256 = wl.random_key(128, 420).tobytes(), wl.random_key(256, 421).tobytes()
        aesgb.aes_srv_put_key(srv, 0, 128, k128)
        aesgb.aes_srv_put_key(srv, 1, 128, k128)
        data = wl.random_bytes(1 << 16, 422)
        x = torch.from_numpy(data).cuda()
        y = torch.full_like(x, 0x5A)
        st, t = aesgb.aes_srv_submit_many(srv, [0], [0], [x.data_ptr()], [y.data_ptr()], [data.size], [30.0])
        assert st == 0
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_put_key(srv, 0, 256, k256)          # the queued request names key 0
        assert e.value.status == -9
        aesgb.aes_srv_put_key(srv, 1, 256, k256)              # key 1 is free to change
        aesgb.aes_srv_cancel(srv, int(t[0]))
        aesgb.aes_srv_put_key(srv, 0, 256, k256)
        t2 = aesgb.aes_srv_submit(srv, 0, 0, x, y, data.size)
        s_, _ = aesgb.aes_srv_wait(srv, t2, 10000)
        assert s_ == 0
        assert np.array_equal(y.cpu().numpy(), orc.ecb(0, k256, data, nthreads=4))
    finally:
        aesgb.aes_srv_destroy(srv)


def test_put_schedule_keeps_expanded_keys(orc):
    """aes_srv_put_schedule takes round keys already expanded (as
    aes_expand_key writes them); requests under them equal the oracle.  A bad
    round count is refused."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(8 << 20, max_keys=3, max_batch=16, slots=2)
    try:
        keys = [wl.random_key(kb, 430 + i).tobytes() for i, kb in enumerate((128, 192, 256))]
        for i, key in enumerate(keys):
            enc, dec, nr = aesgb.aes_expand_key(8 * len(key), key)
            aesgb.aes_srv_put_schedule(srv, i, enc, dec, nr)
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_put_schedule(srv, 0, enc, dec, 13)
        assert e.value.status == -3
        data = wl.random_bytes(3 * 8192, 433)
        x = torch.from_numpy(data).cuda()
        y = torch.full_like(x, 0x5A)
        ts = [aesgb.aes_srv_submit(srv, i, i % 2, x[8192 * i:], y[8192 * i:], 8192) for i in range(3)]
        for t in ts:
            assert aesgb.aes_srv_wait(srv, t, 10000)[0] == 0
        out = y.cpu().numpy()
        for i in range(3):
            w = slice(8192 * i, 8192 * (i + 1))
            assert np.array_equal(out[w], orc.ecb(i % 2, keys[i], data[w])), i
    finally:
        aesgb.aes_srv_destroy(srv)


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
        # a size whose input + output overflows 64 bits: refused, not admitted as 0 bytes
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_submit(srv2, 0, 0, buf, buf, 1 << 63)
        assert e.value.status == -10
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


def test_cancel_queued_requests(orc):
    """Requests still queued (arrival 30 s ahead) are cancelled: they complete
    at once with AES_E_CANCELLED, drain stops waiting for them and their
    outputs are never written.  A request already done cannot be cancelled;
    the ones behind a cancelled request still run and are exact."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(8 << 20, max_keys=1, max_batch=16, slots=2)
    try:
        key = wl.random_key(256, 400).tobytes()
        aesgb.aes_srv_put_key(srv, 0, 256, key)
        sizes = [4096] * 6
        a = Arena(torch, sizes, 401)
        arrivals = [30.0, 0.0, 30.0, 0.0, 30.0, 0.0]
        st, t = aesgb.aes_srv_submit_many(srv, [0] * 6, [0, 1, 0, 1, 0, 1], a.ins(), a.outs(), sizes, arrivals)
        assert st == 0
        for i in (0, 2, 4):
            aesgb.aes_srv_cancel(srv, int(t[i]))
        aesgb.aes_srv_drain(srv, 10000)                          # returns: nothing left to wait for
        status, _, _ = aesgb.aes_srv_results(srv, t)
        assert list(status) == [-13, 0, -13, 0, -13, 0]
        out = a.out.cpu().numpy()
        for i in (0, 2, 4):
            assert np.all(a.msg(out, i) == 0x5A), i
        for i in (1, 3, 5):
            assert np.array_equal(a.msg(out, i), orc.ecb(1, key, a.msg(a.data, i), nthreads=1)), i
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_cancel(srv, int(t[1]))                # done already
        assert e.value.status == -9
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_cancel(srv, 10 ** 9)                  # never issued
        assert e.value.status == -11
        stats = aesgb.aes_srv_stats(srv)
        assert stats["cancelled"] == 3 and stats["completed"] == 6 and stats["bytes_completed"] == 3 * 4096
    finally:
        aesgb.aes_srv_destroy(srv)


def test_registered_ranges_confine_buffers(orc):
    """With a registry, a request is accepted only if its input and output
    each lie inside one registered range (checked on the host before any
    launch); overlapping registrations are refused; an empty registry accepts
    every buffer again."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(8 << 20, max_keys=1, max_batch=16, slots=1)
    try:
        key = wl.random_key(128, 402).tobytes()
        aesgb.aes_srv_put_key(srv, 0, 128, key)
        data = wl.random_bytes(1 << 16, 403)
        n = data.size
        # each registered range is the first half of a larger allocation, so
        # that a request running past it stays inside memory it may touch
        src_all = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
        dst_all = torch.full((2 * n,), 0x5A, dtype=torch.uint8, device="cuda")
        src, dst = src_all[:n], dst_all[:n]
        src.copy_(torch.from_numpy(data))
        other = torch.zeros(n, dtype=torch.uint8, device="cuda")
        aesgb.aes_srv_register(srv, src, n)
        aesgb.aes_srv_register(srv, dst, n)
        for base, size in ((src.data_ptr() + 256, 256), (dst.data_ptr() - 256, 512)):
            with pytest.raises(aesgb.AesError) as e:
                aesgb.aes_srv_register(srv, base, size)          # overlaps a registered range
            assert e.value.status == -5
        refused = [(other.data_ptr(), dst.data_ptr(), 4096),           # input unregistered
                   (src.data_ptr(), other.data_ptr(), 4096),           # output unregistered
                   (src.data_ptr() + n - 4096, dst.data_ptr(), 8192),  # input runs past its range
                   (src.data_ptr(), dst.data_ptr() + 16, n)]           # output runs past its range
        for ip, op, nb in refused:
            with pytest.raises(aesgb.AesError) as e:
                aesgb.aes_srv_submit(srv, 0, 0, ip, op, nb)
            assert e.value.status == -14, (ip - src.data_ptr(), op - dst.data_ptr(), nb)
        t = aesgb.aes_srv_submit(srv, 0, 0, src, dst, n)          # whole ranges: accepted
        s, _ = aesgb.aes_srv_wait(srv, t, 10000)
        assert s == 0
        assert np.array_equal(dst.cpu().numpy(), orc.ecb(0, key, data, nthreads=4))
        aesgb.aes_srv_unregister(srv, src)
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_srv_unregister(srv, src)
        assert e.value.status == -11
        aesgb.aes_srv_unregister(srv, dst)
        t = aesgb.aes_srv_submit(srv, 0, 1, dst, other, n)        # registry empty: any buffer
        s, _ = aesgb.aes_srv_wait(srv, t, 10000)
        assert s == 0 and torch.equal(other, src)
        stats = aesgb.aes_srv_stats(srv)
        assert stats["submitted"] == 2 and stats["worker_status"] == 0
    finally:
        aesgb.aes_srv_destroy(srv)


def test_injected_allocation_failures(orc):
    """Host-side failure injection.  aes_srv_create makes six allocations
    (two key stores, then a page-locked and a device buffer per slot); with
    the k-th of them failing it returns AES_E_NOMEM, frees what it had, and
    the library stays usable.  The library-owned batch workspace, grown for a
    batch larger than any before, reports the same and allocates on the next
    call."""
    torch = torch_cuda()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in range(6):
            aesgb.aes_test_fail_allocs(k, 1)
            with pytest.raises(aesgb.AesError) as e:
                aesgb.aes_srv_create(1 << 20, max_keys=4, max_batch=8, slots=2)
            assert e.value.status == -7, k
        aesgb.aes_test_fail_allocs(0, 0)
        srv = aesgb.aes_srv_create(1 << 20, max_keys=4, max_batch=8, slots=2)
        aesgb.aes_srv_destroy(srv)
        # 200,000 one-block messages of one key: a 4 MB plan, above the
        # 1 MiB workspace the library keeps after small batches
        n = 200_000
        key = wl.random_key(128, 405).tobytes()
        enc, _, nr = aesgb.aes_expand_key(128, key)
        data = wl.random_bytes(16 * n, 406)
        x = torch.from_numpy(data).cuda()
        y = torch.full_like(x, 0x5A)
        rk = torch.from_numpy(enc.view(np.uint8).copy()).cuda()
        off = 16 * np.arange(n, dtype=np.uint64)
        table = aesgb.pack_descs(np.full(n, rk.data_ptr(), np.uint64), x.data_ptr() + off, y.data_ptr() + off,
                                 np.ones(n), np.full(n, nr), np.zeros(n))
        desc = torch.from_numpy(table.view(np.uint8).copy()).cuda()
        aesgb.aes_test_fail_allocs(0, 1)
        with pytest.raises(aesgb.AesError) as e:
            aesgb.aes_ecb_batch(desc, n)
        assert e.value.status == -7
        torch.cuda.synchronize()
        assert bool((y == 0x5A).all())                              # nothing launched
        aesgb.aes_ecb_batch(desc, n)                                # the next call allocates and runs
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), orc.ecb(0, key, data, nthreads=4))
    finally:
        aesgb.aes_test_fail_allocs(0, 0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] > free0 - (64 << 20)       # nothing large leaked



def test_cancel_races_dispatch_under_load(orc):
    """Cancellation racing the dispatcher: 1,500 requests arrive over about
    30 ms while every third one is cancelled right after submission.  Each
    request ends exactly one way: cancelled (AES_E_CANCELLED, output never
    written) or completed bit-exact; the counts add up."""
    torch = torch_cuda()
    srv = aesgb.aes_srv_create(64 << 20, max_keys=4, max_batch=64, slots=3)
    try:
        keys = {}
        g = wl.rng(410)
        for k in range(4):
            kb = (128, 192, 256, 128)[k]
            keys[k] = g.integers(0, 256, kb // 8, dtype=np.uint8).tobytes()
            aesgb.aes_srv_put_key(srv, k, kb, keys[k])
        n = 1500
        sizes = wl.log_uniform_lengths(n, 16, 64 * 1024, g)
        key_ids = g.integers(0, 4, n)
        dirs = g.integers(0, 2, n)
        arrivals = np.sort(g.uniform(0.0, 0.03, n))
        a = Arena(torch, sizes, 411)
        st, t = aesgb.aes_srv_submit_many(srv, key_ids, dirs, a.ins(), a.outs(), sizes, arrivals)
        assert st == 0
        outcome = {}
        for i in range(0, n, 3):
            try:
                aesgb.aes_srv_cancel(srv, int(t[i]))
                outcome[i] = "cancelled"
            except aesgb.AesError as e:
                assert e.status == -9, e.status                      # already launched
                outcome[i] = "launched"
        aesgb.aes_srv_drain(srv, 60000)
        status, _, _ = aesgb.aes_srv_results(srv, t)
        out = a.out.cpu().numpy()
        n_cancelled = 0
        for i in range(n):
            if status[i] == -13:
                assert outcome.get(i) == "cancelled", i
                assert np.all(a.msg(out, i) == 0x5A), i
                n_cancelled += 1
            else:
                assert status[i] == 0 and outcome.get(i) != "cancelled", (i, status[i])
                exp = orc.ecb(int(dirs[i]), keys[int(key_ids[i])], a.msg(a.data, i), nthreads=1)
                assert np.array_equal(a.msg(out, i), exp), i
        stats = aesgb.aes_srv_stats(srv)
        assert stats["cancelled"] == n_cancelled and stats["completed"] == n
        assert stats["bytes_completed"] == int(sizes[status == 0].sum())
        assert 0 < n_cancelled                                            # the race was exercised
    finally:
        aesgb.aes_srv_destroy(srv)
