"""Debug build (AESGB_BOUNDS_CHECK) on small ragged cases: every kernel family
runs with its shared-memory table, tile, mask-plane and key-slot indices and
the global ranges the batch and TMA kernels derive on the device checked.  No
check may fail, no bounded wait may run out, and every result is bit-exact
against the oracle.

The pytest function builds ``libaesgb_debug.so`` and runs this file as a
script in a child process with ``AESGB_LIBRARY=debug`` (the binding chooses its
library once, at import).  The script prints one line per case family and
exits non-zero at the first mismatch or failed check."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.gpu
def test_debug_build_every_kernel_no_failed_check():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_05234_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, AESGB_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    sys.stdout.write(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all cases: 0 failed checks, 0 wait timeouts" in r.stdout


# --------------------------------------------------------------------------
# the child process
# --------------------------------------------------------------------------
def _setup():
    for p in (ROOT, HERE):
        if p not in sys.path:
            sys.path.insert(0, p)
    from paper_1902_05234_gb300 import aesgb
    assert aesgb.LIB_PATH.endswith("libaesgb_debug.so"), aesgb.LIB_PATH
    import oracle
    return aesgb, oracle.Oracle()


def _report(aesgb, what):
    """Read (and reset) both counters after a case family; fail if either is set."""
    import torch
    torch.cuda.synchronize()
    v = aesgb.aes_debug_bounds_violations()
    t = aesgb.aes_wait_timeouts()
    print(f"{what}: {v} failed checks, {t} wait timeouts", flush=True)
    assert v == 0 and t == 0, what


def _ecb_cfgs(aesgb):
    out = []
    for layout in (aesgb.LAYOUT_R4, aesgb.LAYOUT_R1, aesgb.LAYOUT_P4, aesgb.LAYOUT_CONST, aesgb.LAYOUT_R4_TMA,
                   aesgb.LAYOUT_R2, aesgb.LAYOUT_REG):
        nbs = {aesgb.LAYOUT_R4: (1, 2, 4, 8), aesgb.LAYOUT_R2: (1, 2, 4, 8), aesgb.LAYOUT_R1: (1, 2, 4),
               aesgb.LAYOUT_R4_TMA: (1, 2, 4), aesgb.LAYOUT_REG: (1, 2)}.get(layout, (1,))
        for nb in nbs:
            for threads in (64, 256, 512, 1024):
                limit = 256 if (nb == 8 or layout == aesgb.LAYOUT_REG) else 512 if nb == 4 else 1024
                if threads > limit or (threads == 256 and limit > 256):
                    continue
                for cps in (0, 1):
                    out.append(aesgb.make_cfg(threads, nb, layout, cps))
    return out


def run_ecb(aesgb, orc):
    from paper_1902_05234_gb300 import workloads as wl
    from gpu_util import gpu_ecb
    sizes = (1, 33, 1025, 4099)
    cfgs = _ecb_cfgs(aesgb)
    for k, cfg in enumerate(cfgs):
        keybits = (128, 192, 256)[k % 3]
        key = wl.random_key(keybits, 300 + k).tobytes()
        for direction in (0, 1):
            for n in sizes:
                data = wl.random_bytes(16 * n, 310 + n)
                exp = orc.ecb(direction, key, data, nthreads=8)
                got, ok = gpu_ecb(direction, key, data, cfg=cfg, guard=64)
                assert ok and np.array_equal(got, exp), (repr(cfg), direction, n)
            got, ok = gpu_ecb(direction, key, data, cfg=cfg, inplace=True, guard=64)
            assert ok and np.array_equal(got, exp), (repr(cfg), direction, "in place")
    # the tuned default path on every key size
    for keybits in (128, 192, 256):
        key = wl.random_key(keybits, 320).tobytes()
        data = wl.random_bytes(16 * 70_001, 321)
        for direction in (0, 1):
            got, ok = gpu_ecb(direction, key, data, guard=64)
            assert ok and np.array_equal(got, orc.ecb(direction, key, data, nthreads=8)), (keybits, direction)
    _report(aesgb, f"ecb ({len(cfgs)} launch configurations x 2 directions x {len(sizes)} sizes)")


def run_modes_ct_host(aesgb, orc):
    import torch
    from paper_1902_05234_gb300 import workloads as wl
    for keybits in (128, 192, 256):
        key = wl.random_key(keybits, 330).tobytes()
        enc, dec, nr = aesgb.aes_expand_key(keybits, key)
        g = wl.rng(331 + keybits)
        for n in (1, 33, 4097, 70_001):
            data = wl.random_bytes(16 * n, 332 + n)
            iv = g.integers(0, 256, 16, dtype=np.uint8)
            x = torch.from_numpy(data).cuda()
            y = torch.full_like(x, 0x5A)
            aesgb.aes_ctr_crypt(enc, nr, iv, x, y, n)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), orc.ctr(key, iv, data)), ("ctr", keybits, n)
            aesgb.aes_cbc_decrypt(dec, nr, iv, x, y, n)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), orc.cbc_decrypt(key, iv, data)), ("cbc", keybits, n)
            aesgb.aes_cfb_decrypt(enc, nr, iv, x, y, n)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), orc.cfb_decrypt(key, iv, data)), ("cfb", keybits, n)
            for direction, rk in ((0, enc), (1, dec)):
                z = torch.full((16 * n + 64,), 0x5A, dtype=torch.uint8, device="cuda")
                aesgb.aes_ecb_crypt_ct(direction, rk, nr, x, z, n)
                torch.cuda.synchronize()
                got = z.cpu().numpy()
                assert np.array_equal(got[:16 * n], orc.ecb(direction, key, data, nthreads=8)), ("ct", keybits, n)
                assert np.all(got[16 * n:] == 0x5A)
        n = 5001
        data = wl.random_bytes(16 * n, 333)
        h_in = torch.from_numpy(data.copy()).pin_memory()
        h_out = torch.zeros_like(h_in).pin_memory()
        s = torch.cuda.current_stream()
        aesgb.aes_ecb_host_direct(0, enc, nr, h_in, h_out, n, s)
        s.synchronize()
        assert np.array_equal(h_out.numpy(), orc.ecb(0, key, data, nthreads=8)), ("host direct", keybits)
    _report(aesgb, "ctr, cbc / cfb decryption, constant-time, host-direct ECB (3 key sizes x 4 sizes)")


def run_batch(aesgb, orc):
    import torch
    from paper_1902_05234_gb300 import workloads as wl
    from batch_util import DeviceBatch

    def mix(n, hi, seed):
        g = wl.rng(seed)
        return (wl.log_uniform_lengths(n, 16, hi, g), g.choice(np.array([128, 192, 256]), size=n),
                g.integers(0, 2, size=n))

    def expected(b, skip=()):
        return {i: orc.ecb(int(b.dirs[i]), b.keys[i], b.message(b.data, i), nthreads=8)
                for i in range(b.n) if i not in skip}

    def n_chunks(b, cfg, skip=()):
        cb = 32 * cfg.blocks_per_thread * cfg.chunk_passes
        return sum(-(-(int(b.lengths[i]) // 16) // cb) for i in range(b.n) if i not in skip)

    def check_coverage(want, ws=None):
        """Exactly-once: after one launch every chunk of the plan was taken by
        exactly one warp (and the plan's own total, in the workspace header,
        is the host's count)."""
        torch.cuda.synchronize()
        once, repeated, beyond = aesgb.aes_debug_batch_coverage()
        assert (once, repeated, beyond) == (want, 0, 0), (once, repeated, beyond, want)
        if ws is not None:
            assert int(ws[:8].cpu().numpy().view(np.uint64)[0]) == want
        return want

    aesgb.aes_debug_batch_coverage()  # clear

    # invalid descriptors (bad rounds, direction, key pointer, alignment) and a
    # partial overlap: each gets its status and no work, the rest is exact
    lengths, keybits, dirs = mix(200, 64 * 1024, 340)
    lengths[7] = 0
    lengths[15] = 4096
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=341)
    bad = {11: ("nrounds", 11, -3), 12: ("dir", 2, -1), 13: ("rk", 0, -1), 14: ("in", 8, -4)}
    for i, (field, val, _) in bad.items():
        if field == "in":
            b.table[i]["in"] += val
        else:
            b.table[i][field] = val
    b.table[15]["out"] = b.table[15]["in"] + 16
    b.upload()
    ws, nbytes = b.workspace()
    status = torch.full((b.n,), 99, dtype=torch.int32, device="cuda")
    aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, status)
    tagged = check_coverage(n_chunks(b, aesgb.aes_batch_get_cfg(b.n), set(bad) | {15}), ws)
    out, st = b.output(), status.cpu().numpy()
    for i, (_, _, code) in bad.items():
        assert st[i] == code, (i, st[i])
    assert st[15] == -5
    skip = set(bad) | {15}
    for i, exp in expected(b, skip).items():
        assert np.array_equal(b.message(out, i), exp), ("batch with invalid descriptors", i)
    for i in skip:
        assert np.all(b.message(out, i) == 0x5A), ("invalid message written", i)

    # every batch configuration, the library workspace, the no-allocation
    # scratch and a captured graph on one valid mix
    lengths, keybits, dirs = mix(120, 96 * 1024, 342)
    b = DeviceBatch(torch, lengths, keybits, dirs, seed=343)
    exp = np.concatenate([e for _, e in sorted(expected(b).items())])
    ws, nbytes = b.workspace()
    ncfg = 0
    pairs = [(aesgb.LAYOUT_R4, aesgb.LAYOUT_R2, (1, 2, 4)), (aesgb.LAYOUT_R4, aesgb.LAYOUT_R4, (1, 2)),
             (aesgb.LAYOUT_R2, aesgb.LAYOUT_R2, (1, 2)), (aesgb.LAYOUT_R1, aesgb.LAYOUT_R1, (1, 2))]
    cfgs = [aesgb.make_batch_cfg(threads, nb, passes, 1, le, ld)
            for le, ld, nbs in pairs for nb in nbs for threads in (64, 512) for passes in (1, 5)]
    for cfg in cfgs:
        b.out_dev.fill_(0x5A)
        aesgb.aes_ecb_batch_ws(b.desc_dev, b.n, ws, nbytes, cfg=cfg)
        tagged += check_coverage(n_chunks(b, cfg), ws)
        assert np.array_equal(b.output(), exp), ("batch cfg", repr(cfg))
        ncfg += 1
    default = n_chunks(b, aesgb.aes_batch_get_cfg(b.n))
    b.out_dev.fill_(0x5A)
    aesgb.aes_ecb_batch(b.desc_dev, b.n)
    tagged += check_coverage(default)
    assert np.array_equal(b.output(), exp), "library workspace"
    b.out_dev.fill_(0x5A)
    aesgb.aes_ecb_batch_noalloc(b.desc_dev, b.n)
    tagged += check_coverage(default)
    assert np.array_equal(b.output(), exp), "no-allocation scratch"
    graph = aesgb.aes_batch_graph_create(b.desc_dev, b.n, ws, nbytes)
    try:
        for _ in range(2):
            b.out_dev.fill_(0x5A)
            aesgb.aes_batch_graph_launch(graph)
            tagged += check_coverage(default, ws)
            assert np.array_equal(b.output(), exp), "graph replay"
    finally:
        aesgb.aes_batch_graph_destroy(graph)
    _report(aesgb, f"batch (invalid descriptors; {ncfg} configurations; library, no-alloc, graph; "
                   f"{tagged} chunks each taken exactly once)")


def run_server(aesgb, orc):
    import torch
    from paper_1902_05234_gb300 import workloads as wl
    srv = aesgb.aes_srv_create(16 << 20, max_keys=8, max_batch=64, slots=3)
    try:
        keys = {}
        g = wl.rng(350)
        for k in range(8):
            kb = (128, 192, 256)[k % 3]
            keys[k] = g.integers(0, 256, kb // 8, dtype=np.uint8).tobytes()
            aesgb.aes_srv_put_key(srv, k, kb, keys[k])
        n = 150
        sizes = wl.log_uniform_lengths(n, 16, 64 * 1024, g)
        key_ids = g.integers(0, 8, n)
        dirs = g.integers(0, 2, n)
        offs = np.zeros(n + 1, np.int64)
        np.cumsum(sizes, out=offs[1:])
        data = wl.random_bytes(int(offs[-1]), 351)
        inp = torch.from_numpy(data).cuda()
        outp = torch.full_like(inp, 0x5A)
        ins = inp.data_ptr() + offs[:-1].astype(np.uint64)
        outs = outp.data_ptr() + offs[:-1].astype(np.uint64)
        st, tickets = aesgb.aes_srv_submit_many(srv, key_ids, dirs, ins, outs, sizes)
        assert st == 0
        aesgb.aes_srv_drain(srv, 60000)
        status, _, _ = aesgb.aes_srv_results(srv, tickets, release=True)
        assert np.all(status == 0)
        got = outp.cpu().numpy()
        for i in range(n):
            exp = orc.ecb(int(dirs[i]), keys[int(key_ids[i])], data[offs[i]:offs[i + 1]], nthreads=1)
            assert np.array_equal(got[offs[i]:offs[i + 1]], exp), ("served", i)
    finally:
        aesgb.aes_srv_destroy(srv)
    _report(aesgb, f"server ({n} requests, 8 keys)")


def main():
    aesgb, orc = _setup()
    # only the debug library answers AES_OK here (the release build raises
    # AES_E_CONFIG); nothing has run yet, so both counters start at zero
    assert aesgb.aes_debug_bounds_violations() == 0
    assert aesgb.aes_wait_timeouts() == 0
    run_ecb(aesgb, orc)
    run_modes_ct_host(aesgb, orc)
    run_batch(aesgb, orc)
    run_server(aesgb, orc)
    print("all cases: 0 failed checks, 0 wait timeouts", flush=True)


if __name__ == "__main__":
    main()
