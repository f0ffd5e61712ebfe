#!/usr/bin/env python3
"""Benchmark of the GB300 bulk AES library (one JSON line on rank 0).

Workload of a step (per rank, weak scaling): AES-128 ECB over a 1 GiB buffer of
seeded uniform random bytes already resident in HBM -- the host key schedule
(aes_expand_key), encryption of the buffer into a second buffer, decryption of
that ciphertext into a third -- i.e. every step of the single-buffer hot path in
both directions.  `value` is Gbit/s of plaintext+ciphertext processed (2 GiB per
rank per step), device-timed with CUDA events on the launching stream, the max
over ranks.  Inputs (1 GiB) are larger than the 129 MB L2, so no flush is needed.

Additional objects on the same line:
  roofline     the encryption kernel against its bound, the shared-memory lookup
               rate (16 lookups of 4 B per block per round; 32 lanes x 4 B per clock
               per SM), at the SM clock sampled during the timed region.
  e2e          the same two passes through aes_ecb_host_direct on page-locked host
               buffers: the kernel itself reads the input from and writes the output to
               host memory, so every byte crosses the host link inside the timed region.
  cpu_baseline the CPU oracle timed on this host's cores on a bounded sample.
  sweep        single-buffer Gbit/s over 1 MiB..4 GiB x AES-128/192/256 x enc/dec.
  clocks       nvidia-smi SM clock and throttle reasons sampled while timing.

`--impl reference` times the CPU oracle instead (the reference arm of this
method is the plain FIPS-197 CPU implementation), on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GIB = 1 << 30
MIB = 1 << 20
METRIC = "AES-128 ECB enc/dec throughput (single 1 GiB buffer, HBM-resident)"
UNIT = "Gbit/s"
KERNEL_SOURCES = ["paper_1902_05234_gb300/csrc/aes_kernels.cuh",
                  "paper_1902_05234_gb300/csrc/aes_tables.h",
                  "paper_1902_05234_gb300/csrc/bounds.cuh"]


def parse_args():
    p = argparse.ArgumentParser(
        description="Bulk AES ECB on one or more GB300s: one JSON line with the timed throughput, its roofline, "
                    "the end-to-end figure, the other sections and the CPU oracle baseline.")
    p.add_argument("--gpus", type=int, default=1, help="GPUs (one process each under torchrun; replicas)")
    p.add_argument("--steps", type=int, default=200, help="timed steps (one encrypt + one decrypt launch each)")
    p.add_argument("--warmup", type=int, default=5, help="untimed warm-up steps before the timed ones")
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300",
                   help="gb300: the CUDA kernels; reference: the CPU oracle on this host's cores")
    p.add_argument("--bytes", type=int, default=GIB, help="buffer size per rank")
    p.add_argument("--keybits", type=int, default=128, help="AES key size of the timed workload (128, 192, 256)")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (end-to-end) measurement")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-sweep", action="store_true", help="skip the size x key size x direction sweep")
    p.add_argument("--no-batched", action="store_true", help="skip the batched (descriptor table) section")
    p.add_argument("--no-served", action="store_true", help="skip the continuous-batching server section")
    p.add_argument("--no-tune", action="store_true", help="time the default launch configurations, no autotuning")
    p.add_argument("--no-stress", action="store_true", help="skip the 16 GiB in-place AES-256 decryption")
    p.add_argument("--no-ct", action="store_true", help="skip the constant-time (bitsliced) kernel")
    p.add_argument("--served-requests", type=int, default=20000, help="requests per load point of the served sweep")
    p.add_argument("--served-slots", type=int, default=4, help="in-flight batch slots of the served section's server")
    p.add_argument("--batch-n", type=int, default=4096, help="messages in the batched workload")
    p.add_argument("--batch-max-bytes", type=int, default=16 * MIB, help="largest message of the batched workload")
    p.add_argument("--study", action="store_true",
                   help="placement / granularity study (the paper's section 4 design axis) instead of the bench")
    p.add_argument("--study-reps", type=int, default=5, help="timed repetitions per study variant")
    p.add_argument("--study-dir", type=int, choices=[0, 1], default=0,
                   help="direction of the study's runs: 0 encrypt, 1 decrypt")
    p.add_argument("--study-warmup", type=int, default=2, help="warm-up repetitions per study variant")
    return p.parse_args()


def workload_config(args, world):
    return {
        "workload": f"AES-{args.keybits} ECB encrypt then decrypt of one {args.bytes // MIB} MiB buffer "
                    f"({args.bytes // 16:,} blocks) per GPU, uniform random bytes, one random key",
        "key_bits": args.keybits,
        "buffer_bytes": args.bytes,
        "mode": "ECB",
        "l2": "inputs larger than L2 (buffer > 129 MB), no flush",
        "parallelism": f"independent shards x{world}" if world > 1 else "single GPU",
    }


# ---------------------------------------------------------------------------
# distributed plumbing (timing barrier and max over ranks only)
# ---------------------------------------------------------------------------

class Dist:
    """Host-side process group of a multi-GPU run (gloo: barriers and the
    max / sum over ranks only; no data is exchanged).  Every collective is
    bounded by `timeout_s`: a rank that died or never arrives makes the others'
    next collective raise instead of hang."""

    def __init__(self, timeout_s: float = 600.0):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import datetime
            import torch.distributed as dist
            dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=timeout_s))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate_throughput(dist: "Dist", local_ms: float, local_bits: float, steps: int):
    """Whole-job numbers of a weak-scaling run: every rank processed its own
    shard (`local_bits` per step, no data exchanged); the job's time is the
    slowest rank's, its work the sum over ranks.  Returns (ms_per_step,
    Gbit/s of the whole job)."""
    max_ms = dist.max(local_ms)
    bits = dist.sum(local_bits)
    ms_per_step = max_ms / steps
    return ms_per_step, bits / (ms_per_step / 1e3) / 1e9


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        time.sleep(0.25)  # first sample before the timed work starts

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.REASONS, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, keybits: int, nbytes: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if (kv.get("kernel") == kernel and kv.get("src") == want and int(kv.get("keybits", 0)) == keybits
                and int(kv.get("buffer_bytes", 0)) == nbytes):
            return int(kv["dram_bytes_per_launch"])
    return None


def nrounds_of(keybits: int) -> int:
    return {128: 10, 192: 12, 256: 14}[keybits]


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def oracle_rate(o, nthreads: int) -> float:
    """Bytes/s of the oracle (encrypt) on this host, from a short probe."""
    from paper_1902_05234_gb300 import workloads as wl
    data = wl.random_bytes(256 * 1024, 90)
    key = wl.random_key(128, 90).tobytes()
    t = time.perf_counter()
    o.ecb(0, key, data, nthreads=nthreads)
    return data.size / max(time.perf_counter() - t, 1e-6)


def openssl_speed():
    """Context only: OpenSSL's AES-128-ECB (hardware AES instructions) on one
    host core, if the openssl program exists on this host."""
    import shutil
    exe = shutil.which("openssl")
    if not exe:
        return None
    try:
        r = subprocess.run([exe, "speed", "-elapsed", "-seconds", "1", "-evp", "aes-128-ecb"],
                           capture_output=True, text=True, timeout=60)
    except (OSError, subprocess.TimeoutExpired):
        return None
    for line in r.stdout.splitlines()[::-1]:
        parts = line.split()
        if parts and parts[0].lower().startswith("aes-128"):
            try:
                kbs = float(parts[-1].rstrip("k"))  # largest block size, 1000s of bytes per second
            except ValueError:
                return None
            return {"gbps_one_core": round(kbs * 1000 * 8 / 1e9, 2), "source": "openssl speed -evp aes-128-ecb",
                    "note": "context: hardware AES instructions on one host core, not the oracle"}
    return None


def cpu_baseline(keybits: int, seconds: float = 10.0) -> dict:
    """The oracle as it stands, encrypt + decrypt of a seeded sample sized to
    take about `seconds` on all host cores."""
    import oracle
    from paper_1902_05234_gb300 import workloads as wl
    o = oracle.Oracle()
    cores = os.cpu_count() or 1
    rate = oracle_rate(o, cores)
    nbytes = int(min(64 * MIB, max(MIB, rate * seconds / 2))) // 16 * 16
    data = wl.random_bytes(nbytes, 91)
    key = wl.random_key(keybits, 91).tobytes()
    t0 = time.perf_counter()
    ct = o.ecb(0, key, data, nthreads=cores)
    t1 = time.perf_counter()
    o.ecb(1, key, ct, nthreads=cores)
    t2 = time.perf_counter()
    gbps = 2 * nbytes * 8 / (t2 - t0) / 1e9
    # one thread on 1 MiB, for the per-core figure
    small = data[:MIB]
    t3 = time.perf_counter()
    o.ecb(0, key, small, nthreads=1)
    single = small.size * 8 / (time.perf_counter() - t3) / 1e9
    # every key size and direction: all cores on the sample and on 1 MiB, one
    # thread on 1 MiB (about 10 s more in all)
    by_key = {}
    for kb in (128, 192, 256):
        k = wl.random_key(kb, 92).tobytes()
        row = {}
        for d, name in ((0, "enc"), (1, "dec")):
            cell = {}
            for label, buf, nt in (("all_cores_sample", data, cores), ("all_cores_1MiB", small, cores),
                                   ("single_thread_1MiB", small, 1)):
                t = time.perf_counter()
                o.ecb(d, k, buf, nthreads=nt)
                cell[label] = round(buf.size * 8 / (time.perf_counter() - t) / 1e9, 5)
            row[name] = cell
        by_key[str(kb)] = row
    return {"value": gbps, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_gbps": round(single, 5), "by_key": by_key, "openssl_context": openssl_speed(),
            "sample": f"AES-{keybits} ECB encrypt+decrypt of {nbytes:,} bytes (seeded uniform random), "
                      f"{cores} threads, contiguous split",
            "seconds": round(t2 - t0, 3), "enc_s": round(t1 - t0, 3), "dec_s": round(t2 - t1, 3)}


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return
    import oracle
    from paper_1902_05234_gb300 import workloads as wl
    o = oracle.Oracle()
    cores = os.cpu_count() or 1
    rate = oracle_rate(o, cores)
    budget_s = min(2.0, 150.0 / max(1, args.steps + args.warmup))
    nbytes = max(16 * 1024, int(rate * budget_s / 2) // 16 * 16)
    data = wl.random_bytes(nbytes, 92)
    key = wl.random_key(args.keybits, 92).tobytes()
    for _ in range(args.warmup):
        o.ecb(1, key, o.ecb(0, key, data, nthreads=cores), nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.ecb(1, key, o.ecb(0, key, data, nthreads=cores), nthreads=cores)
    dt = time.perf_counter() - t
    ms = dt / args.steps * 1e3
    gbps = 2 * nbytes * 8 * args.steps / dt / 1e9
    sample = (f"each step: AES-{args.keybits} ECB encrypt+decrypt of {nbytes:,} bytes of the workload's "
              f"distribution on {cores} host threads")
    line = {"metric": METRIC, "value": gbps, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args, args.gpus),
            "cpu_baseline": {"value": gbps, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------

def timed_ecb(torch, aesgb, rk, nr, direction, src, dst, nblocks, iters=5, warm=2, replays=5):
    """Device time of one launch.  Small buffers take a few microseconds, less
    than a Python call, so the launches are captured in a CUDA graph and the
    replay is timed: the GPU then runs them back to back.  The median of
    `replays` timed replays is taken, so one disturbed replay does not decide
    a microsecond-scale point."""
    fn = aesgb.aes_ecb_encrypt if direction == 0 else aesgb.aes_ecb_decrypt
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        for _ in range(warm):
            fn(rk, nr, src, dst, nblocks, cap)
    cap.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        for _ in range(iters):
            fn(rk, nr, src, dst, nblocks, cap)
    g.replay()
    torch.cuda.synchronize()
    times = []
    for _ in range(replays):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        g.replay()
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e) / iters)
    del g
    return statistics.median(times)


def run_sweep(torch, aesgb, dev, tune=True):
    """Single-buffer sweep: 1 MiB .. 4 GiB (powers of 4) x key sizes x directions,
    each point tuned first (untimed) as a deployment would."""
    from paper_1902_05234_gb300 import workloads as wl
    sizes = [MIB * 4 ** i for i in range(7)]
    big = sizes[-1]
    src = torch.empty(big, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 20)
    src.random_(0, 256, generator=g)
    dst = torch.empty_like(src)
    rows = []
    for kb in (128, 192, 256):
        enc, dec, nr = aesgb.aes_expand_key(kb, wl.random_key(kb, 20).tobytes())
        for d in (0, 1):
            for sz in sizes:
                n = sz // 16
                rk = enc if d == 0 else dec
                cfg = aesgb.aes_tune_ecb(d, nr, rk, src, dst, n) if tune else aesgb.aes_ecb_get_cfg(d, nr, n)
                iters = 5 if sz >= 256 * MIB else 50
                ms = timed_ecb(torch, aesgb, rk, nr, d, src, dst, n, iters=iters)
                rows.append({"keybits": kb, "dir": "enc" if d == 0 else "dec", "bytes": sz,
                             "ms": round(ms, 4), "gbps": round(sz * 8 / ms / 1e6, 1), "cfg": repr(cfg)})
    del src, dst
    torch.cuda.empty_cache()
    return rows


def run_batched(torch, aesgb, dev, n=4096, tune=True, hi=16 * MIB):
    """Batched workload: 4,096 messages, log-uniform 16 B .. 16 MiB, key size
    uniform over {128,192,256}, direction 50/50 -- one persistent launch from a
    device descriptor table replayed as a CUDA graph, against the same messages
    as one aes_ecb_encrypt/decrypt launch each (the loop a user of the plain
    API writes), both as a CUDA-graph replay of the launches and as a Python
    loop with the key schedule per message."""
    import numpy as np
    from paper_1902_05234_gb300 import workloads as wl
    lengths, keybits, dirs = wl.batch_workload(n, hi=hi)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=offs[1:])
    total = int(offs[-1])
    src = torch.empty(total, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 40)
    src.random_(0, 256, generator=g)
    dst = torch.empty_like(src)
    ref = torch.empty_like(src)
    kg = wl.rng(40)
    keys = [kg.integers(0, 256, int(kb) // 8, dtype=np.uint8).tobytes() for kb in keybits]
    rks = np.zeros((n, 64), np.uint32)
    host_rk, nrs = [], np.zeros(n, np.int64)
    for i in range(n):
        enc, dec, nr = aesgb.aes_expand_key(int(keybits[i]), keys[i])
        rk = enc if dirs[i] == 0 else dec
        rks[i, :60] = rk
        host_rk.append(rk)
        nrs[i] = nr
    rk_dev = torch.from_numpy(rks.view(np.uint8).reshape(-1)).to(dev)
    table = aesgb.pack_descs(rk_dev.data_ptr() + 256 * np.arange(n, dtype=np.uint64),
                             src.data_ptr() + offs[:-1].astype(np.uint64),
                             dst.data_ptr() + offs[:-1].astype(np.uint64), lengths // 16, nrs, dirs)
    desc = torch.from_numpy(table.view(np.uint8).copy()).to(dev)
    ws_bytes = aesgb.aes_batch_workspace_bytes(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def ev_time(fn, iters):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(stream)
        for _ in range(iters):
            fn()
        e_.record(stream)
        e_.synchronize()
        return s_.elapsed_time(e_) / iters

    tuned = repr(aesgb.aes_tune_batch(desc, n, ws, ws_bytes, stream)) if tune else None
    graph = aesgb.aes_batch_graph_create(desc, n, ws, ws_bytes)
    try:
        for _ in range(2):
            aesgb.aes_batch_graph_launch(graph, stream)
        ms_batch = ev_time(lambda: aesgb.aes_batch_graph_launch(graph, stream), 5)
    finally:
        aesgb.aes_batch_graph_destroy(graph)

    def loop_launches(strm):
        for i in range(n):
            nb = int(lengths[i]) // 16
            a, b = src.data_ptr() + int(offs[i]), ref.data_ptr() + int(offs[i])
            if dirs[i] == 0:
                aesgb.aes_ecb_encrypt(host_rk[i], int(nrs[i]), a, b, nb, strm)
            else:
                aesgb.aes_ecb_decrypt(host_rk[i], int(nrs[i]), a, b, nb, strm)

    loop_launches(stream)
    torch.cuda.synchronize()
    same = bool(torch.equal(dst, ref))
    cap = torch.cuda.Stream()
    lg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(lg, stream=cap, capture_error_mode="relaxed"):
        loop_launches(cap)
    lg.replay()
    torch.cuda.synchronize()
    ms_loop_graph = ev_time(lg.replay, 3)
    del lg

    def py_loop():
        for i in range(n):
            enc, dec, nr = aesgb.aes_expand_key(int(keybits[i]), keys[i])
            nb = int(lengths[i]) // 16
            a, b = src.data_ptr() + int(offs[i]), ref.data_ptr() + int(offs[i])
            if dirs[i] == 0:
                aesgb.aes_ecb_encrypt(enc, nr, a, b, nb, stream)
            else:
                aesgb.aes_ecb_decrypt(dec, nr, a, b, nb, stream)
    py_loop()
    torch.cuda.synchronize()
    t = time.perf_counter()
    py_loop()
    torch.cuda.synchronize()
    ms_loop_py = (time.perf_counter() - t) * 1e3
    gb = total * 8 / 1e9
    out = {"workload": f"{n} messages, log-uniform 16 B..{hi // MIB} MiB (total {total:,} B), keys uniform over "
                       f"128/192/256, direction 50/50",
           "total_bytes": total, "ms": round(ms_batch, 4), "gbps": round(gb / (ms_batch / 1e3), 1),
           "loop_graph_ms": round(ms_loop_graph, 4), "loop_graph_gbps": round(gb / (ms_loop_graph / 1e3), 1),
           "loop_python_ms": round(ms_loop_py, 3), "loop_python_gbps": round(gb / (ms_loop_py / 1e3), 1),
           "speedup_vs_loop_graph": round(ms_loop_graph / ms_batch, 3),
           "speedup_vs_loop_python": round(ms_loop_py / ms_batch, 3),
           "identical_to_loop": same, "cfg": repr(aesgb.aes_batch_get_cfg(n)), "tuned": tuned is not None}
    del src, dst, ref, rk_dev, desc, ws
    torch.cuda.empty_cache()
    return out


def batch_roofline(batched, n, hi, sms, f_mhz):
    """The single-buffer kernel's bounds summed over the batch's messages: a
    block of a message with Nr rounds moves 64 Nr + 32 bytes through the
    L1TEX data pipe (16 Nr four-byte lookups, a 16-byte load and store), which
    serves 128 B per clock per SM; the lookups alone (64 Nr bytes) give the
    shared-memory bound."""
    from paper_1902_05234_gb300 import workloads as wl
    lengths, keybits, _ = wl.batch_workload(n, hi=hi)
    blocks = lengths.astype(float) / 16
    nr = keybits.astype(float) / 32 + 6
    rate = sms * 128 * f_mhz * 1e6  # bytes per second through the pipe
    bits = float(lengths.sum()) * 8
    l1 = bits / (float((blocks * (64 * nr + 32)).sum()) / rate) / 1e9
    smem = bits / (float((blocks * 64 * nr).sum()) / rate) / 1e9
    return {"bound": "l1tex", "unit": "Gbit/s", "peak": round(l1, 1), "frac": round(batched["gbps"] / l1, 4),
            "smem_peak": round(smem, 1), "smem_frac": round(batched["gbps"] / smem, 4),
            "peak_basis": f"{sms} SMs x {f_mhz:.0f} MHz x 128 B/clk over 64 Nr + 32 B per block of each message"}


def run_served(torch, aesgb, dev, n_req=20000, loads=(0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0), slots=4):
    """Served workload: a Poisson stream of encrypt/decrypt requests, sizes
    log-uniform 64 B .. 4 MiB, keys drawn from 1,024 resident schedules,
    direction 50/50, through the continuous-batching server under a 4 GiB
    device-memory budget.  Peak = the same requests all arriving at once;
    offered load is then swept as a fraction of that peak.  The peak is set
    against the same requests as one plain launch each (served_loop_baseline)."""
    import numpy as np
    from paper_1902_05234_gb300 import workloads as wl
    unit_arrivals, sizes, key_ids, dirs = wl.served_workload(n_req, rate_per_s=1.0, n_keys=1024)
    offs = np.zeros(n_req + 1, np.int64)
    np.cumsum(sizes, out=offs[1:])
    total = int(offs[-1])
    src = torch.empty(total, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 60)
    src.random_(0, 256, generator=g)
    dst = torch.empty_like(src)
    ins = src.data_ptr() + offs[:-1].astype(np.uint64)
    outs = dst.data_ptr() + offs[:-1].astype(np.uint64)
    srv = aesgb.aes_srv_create(4 << 30, 1024, max_batch=8192, slots=slots)
    try:
        kg = wl.rng(61)
        host_keys = []
        for k in range(1024):
            kb = int(kg.choice([128, 192, 256]))
            host_keys.append((kb, kg.integers(0, 256, kb // 8, dtype=np.uint8).tobytes()))
            aesgb.aes_srv_put_key(srv, k, *host_keys[-1])

        submit_ms = []

        def run(offsets):
            t_sub = time.perf_counter()
            st, tickets = aesgb.aes_srv_submit_many(srv, key_ids, dirs, ins, outs, sizes, offsets)
            submit_ms.append((time.perf_counter() - t_sub) * 1e3)
            if st != 0:
                raise SystemExit(f"served: submission refused ({st})")
            aesgb.aes_srv_drain(srv, 600000)
            status, lat, queue = aesgb.aes_srv_results(srv, tickets, release=True)
            if not np.all(status == 0):
                raise SystemExit("served: a request failed")
            arr = offsets if offsets is not None else np.zeros(n_req)
            span = float(np.max(arr + lat) - np.min(arr))
            return lat, queue, span

        run(None)                                   # warm-up (tuned configuration, first launches)
        ref = dst.clone()
        # saturated: every request at once; the peak is the best of three
        peak_bps = max(total / run(None)[2] for _ in range(3))
        rows = []
        identical = bool(torch.equal(dst, ref))
        mean_size = float(np.mean(sizes))
        for load in loads:
            rate = load * peak_bps / mean_size
            offsets = unit_arrivals / rate
            offsets = offsets - offsets[0]
            lat, queue, span = run(offsets)
            identical = identical and bool(torch.equal(dst, ref))
            rows.append({"load": load, "offered_gbps": round(load * peak_bps * 8 / 1e9, 1),
                         "gbps": round(total * 8 / span / 1e9, 1),
                         "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 4),
                         "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 4),
                         "p99_queue_ms": round(float(np.percentile(queue, 99)) * 1e3, 4)})
        # one more saturated pass with device timing on (off above: its events
        # add about 10 us to a light-load request), for the batches' overlap
        aesgb.aes_srv_set_device_timing(srv, True)
        timed_gbps = total * 8 / run(None)[2] / 1e9
        stats = aesgb.aes_srv_stats(srv)
    finally:
        aesgb.aes_srv_destroy(srv)
    loop = served_loop_baseline(torch, aesgb, src, ref, offs, sizes, key_ids, dirs, host_keys)
    out = {"workload": f"{n_req} requests per load point, Poisson arrivals, sizes log-uniform 64 B..4 MiB "
                       f"(total {total:,} B), 1,024 resident keys (128/192/256), direction 50/50, "
                       f"4 GiB budget, {slots} in-flight batches",
           "peak_gbps": round(peak_bps * 8 / 1e9, 1), "sweep": rows,
           "submit_many_ms": round(statistics.median(submit_ms), 3),
           "identical_across_loads": identical, "batches_total": stats["batches"],
           "peak_inflight_bytes": stats["peak_inflight_bytes"],
           "peak_busy_slots": stats["peak_busy_slots"],
           "device_timing": {"peak_device_batches": stats["peak_device_batches"],
                             "device_overlap_s": round(stats["device_overlap_s"], 4),
                             "timed_batches": stats["timed_batches"], "saturated_gbps": round(timed_gbps, 1)},
           "loop_graph_gbps": loop["graph_gbps"], "loop_python_gbps": loop["python_gbps"],
           "speedup_vs_loop_graph": round(peak_bps * 8 / 1e9 / loop["graph_gbps"], 3),
           "speedup_vs_loop_python": round(peak_bps * 8 / 1e9 / loop["python_gbps"], 3),
           "identical_to_loop": loop["identical"]}
    del src, dst, ref
    torch.cuda.empty_cache()
    return out


def served_loop_baseline(torch, aesgb, src, ref, offs, sizes, key_ids, dirs, host_keys):
    """The served requests as the loop a caller writes without the server: one
    aes_ecb_encrypt/decrypt launch per request on one stream, schedules
    expanded on the host beforehand.  Timed as a Python loop (launch overhead
    included, as the caller would see it) and as a CUDA-graph replay of the
    same launches (the launch cost taken away); the output must equal the
    server's."""
    import numpy as np
    n = len(sizes)
    total = int(offs[-1])
    out = torch.empty_like(src)
    sched = [aesgb.aes_expand_key(kb, key) for kb, key in host_keys]
    stream = torch.cuda.current_stream()
    ins = [src.data_ptr() + int(offs[i]) for i in range(n)]
    outs = [out.data_ptr() + int(offs[i]) for i in range(n)]

    def launches(strm):
        for i in range(n):
            enc, dec, nr = sched[int(key_ids[i])]
            if dirs[i] == 0:
                aesgb.aes_ecb_encrypt(enc, nr, ins[i], outs[i], int(sizes[i]) // 16, strm)
            else:
                aesgb.aes_ecb_decrypt(dec, nr, ins[i], outs[i], int(sizes[i]) // 16, strm)

    launches(stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    launches(stream)
    torch.cuda.synchronize()
    py_s = time.perf_counter() - t
    identical = bool(torch.equal(out, ref))
    cap = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
        launches(cap)
    g.replay()
    torch.cuda.synchronize()
    s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_.record(stream)
    for _ in range(3):
        g.replay()
    e_.record(stream)
    e_.synchronize()
    graph_s = s_.elapsed_time(e_) / 3 / 1e3
    del g, out
    return {"graph_gbps": round(total * 8 / graph_s / 1e9, 1), "python_gbps": round(total * 8 / py_s / 1e9, 1),
            "identical": identical}


STUDY_VARIANTS = [  # (label, layout, blocks/thread, threads)
    ("constant memory (paper 4.2), 16 B/thread", 3, 1, 256),
    ("shared, 4 plain tables, 16 B/thread", 2, 1, 1024),
    ("shared, 1 replicated table + rotations, 16 B/thread", 1, 1, 1024),
    ("shared, 1 replicated table + rotations, 32 B/thread", 1, 2, 1024),
    ("shared, 4 replicated tables, 16 B/thread", 0, 1, 1024),
    ("shared, 4 replicated tables, 32 B/thread", 0, 2, 1024),
    ("shared, 4 replicated tables, 64 B/thread", 0, 4, 512),
    ("shared, 4 replicated tables, TMA-staged input, 32 B/thread", 4, 2, 1024),
    ("shared, 4 replicated tables, TMA-staged input, 64 B/thread", 4, 4, 512),
    ("shared, 2 replicated tables + one rotation per column, 16 B/thread", 5, 1, 1024),
    ("shared, 2 replicated tables + one rotation per column, 32 B/thread", 5, 2, 1024),
    ("shared, 2 replicated tables + one rotation per column, 64 B/thread", 5, 4, 512),
    ("shared, 4 replicated tables, 128 B/thread", 0, 8, 256),
    ("shared, 2 replicated tables + one rotation per column, 128 B/thread", 5, 8, 256),
    ("registers, T0 spread over the warp's lanes, shuffles + selects, 16 B/thread", 6, 1, 256),
    ("registers, T0 spread over the warp's lanes, shuffles + selects, 32 B/thread", 6, 2, 256),
]


def run_study(args):
    """Every table placement and granularity on one AES-128 encryption (or,
    with --study-dir 1, decryption) of --bytes, each launched --study-warmup +
    --study-reps times (1 + 0 under ncu gives one launch per variant, in the
    order listed)."""
    import torch
    from paper_1902_05234_gb300 import aesgb
    from paper_1902_05234_gb300 import workloads as wl
    torch.cuda.set_device(0)
    nbytes = args.bytes // 16 * 16
    n = nbytes // 16
    x = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.BASE_SEED + 100)
    x.random_(0, 256, generator=g)
    y = torch.empty_like(x)
    ref = torch.empty_like(x)
    enc, dec, nr = aesgb.aes_expand_key(128, wl.random_key(128, 100).tobytes())
    d = args.study_dir
    rk = enc if d == 0 else dec
    rows = []
    variants = STUDY_VARIANTS + [("constant time: bitsliced, no tables, 32 blocks per thread", None, 32, 256)]
    for i, (label, layout, nb, threads) in enumerate(variants):
        if layout is None:
            cfg = "aes_ecb_crypt_ct(threads=256, 32 blocks/thread)"
            launch = lambda: aesgb.aes_ecb_crypt_ct(d, rk, nr, x, y, n)  # noqa: E731
        else:
            cfg = aesgb.make_cfg(threads, nb, layout, 0)
            launch = lambda c=cfg: aesgb.aes_ecb_crypt_cfg(d, rk, nr, x, y, n, c)  # noqa: E731
        for _ in range(args.study_warmup):
            launch()
        ms = None
        if args.study_reps > 0:
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(args.study_reps):
                launch()
            e.record()
            e.synchronize()
            ms = s.elapsed_time(e) / args.study_reps
        torch.cuda.synchronize()
        if i == 0:
            ref.copy_(y)
        rows.append({"variant": label, "cfg": cfg if isinstance(cfg, str) else repr(cfg),
                     "ms": None if ms is None else round(ms, 4),
                     "gbps": None if ms is None else round(nbytes * 8 / ms / 1e6, 1),
                     "same_output": bool(torch.equal(y, ref))})
    print(json.dumps({"study": "AES-128 ECB " + ("encryption" if d == 0 else "decryption") +
                      ", table placement x granularity",
                      "bytes": nbytes, "rows": rows}), flush=True)


def run_constant_time(torch, aesgb, src, nbytes, key, keybits, iters=5):
    """The bitsliced (table-free, constant-time) kernel on the same buffer,
    both directions and every key size, checked equal to the T-table
    kernel's output.  `enc` / `dec` are the run's own key size; `by_key`
    holds all three (the key of each size is the run's key, cut or
    extended)."""
    n = nbytes // 16
    out = {"by_key": {}}
    dst = torch.empty_like(src)
    ref = torch.empty_like(src)
    for kb in (128, 192, 256):
        k = (key * 2)[:kb // 8]
        enc, dec, nr = aesgb.aes_expand_key(kb, k)
        aesgb.aes_ecb_encrypt(enc, nr, src, ref, n)
        res = {}
        for d, rk, name in ((0, enc, "enc"), (1, dec, "dec")):
            a, b = (src, dst) if d == 0 else (ref, dst)
            aesgb.aes_ecb_crypt_ct(d, rk, nr, a, b, n)
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record()
            for _ in range(iters):
                aesgb.aes_ecb_crypt_ct(d, rk, nr, a, b, n)
            e_.record()
            e_.synchronize()
            ms = s_.elapsed_time(e_) / iters
            same = bool(torch.equal(b, ref if d == 0 else src))
            res[name] = {"ms": round(ms, 4), "gbps": round(nbytes * 8 / ms / 1e6, 1), "same_as_table_path": same}
        out["by_key"][str(kb)] = res
        if kb == keybits:
            out.update(res)
    del ref, dst
    torch.cuda.empty_cache()
    return {"workload": f"AES-{keybits} ECB, {nbytes // MIB} MiB, bitsliced (no table lookups)", **out}


def ct_roofline(aesgb, ct, nbytes, keybits, sms, f_mhz, logic_cal=None):
    """The bitsliced kernel is bound by the integer-logic (ALU) pipe: 64 lanes
    per clock per SM, one 3-input gate or byte permute per lane.  achieved =
    the logic operations its circuits spend per block (aes_ct_ops_per_block,
    counted from the gate tables) x blocks per second; peak = SMs x 64 x the
    SM clock sampled under load.  logic_cal = (ops, seconds) of the LOP3
    calibration kernel, the measured counterpart of the 64."""
    nr = nrounds_of(keybits)
    peak = sms * 64 * f_mhz * 1e6 / 1e12
    out = {"bound": "alu", "unit": "Tops/s", "peak": round(peak, 2),
           "peak_basis": f"{sms} SMs x 64 logic lanes/clk x {f_mhz:.0f} MHz (median sampled under load)"}
    if logic_cal is not None:
        ops, secs = logic_cal
        out["measured_peak"] = {"tops": round(ops / secs / 1e12, 2),
                                "lanes_per_clk_per_sm": round(ops / secs / (sms * f_mhz * 1e6), 2),
                                "source": "aes_calibrate_logic_rate (8 independent LOP3 chains per thread)"}
    for d, name in ((0, "enc"), (1, "dec")):
        ops = aesgb.aes_ct_ops_per_block(d, nr)
        achieved = ops * (nbytes / 16) / (ct[name]["ms"] / 1e3) / 1e12
        out[name] = {"ops_per_block": round(ops, 2), "achieved": round(achieved, 2), "frac": round(achieved / peak, 4)}
        if logic_cal is not None:
            out[name]["measured_frac"] = round(achieved / (logic_cal[0] / logic_cal[1] / 1e12), 4)
    return out


def run_modes(torch, aesgb, src, nbytes, key, keybits, iters=5):
    """CTR and parallel CBC / CFB decryption on the same buffer (same tables
    and round code as ECB, so the same shared-memory lookup bound)."""
    n = nbytes // 16
    enc, dec, nr = aesgb.aes_expand_key(keybits, key)
    dst = torch.empty_like(src)
    out = {}
    iv = bytes(range(16))
    for name, fn in (("ctr", lambda: aesgb.aes_ctr_crypt(enc, nr, iv, src, dst, n)),
                     ("cbc_decrypt", lambda: aesgb.aes_cbc_decrypt(dec, nr, iv, src, dst, n)),
                     ("cfb_decrypt", lambda: aesgb.aes_cfb_decrypt(enc, nr, iv, src, dst, n))):
        fn()
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record()
        for _ in range(iters):
            fn()
        e_.record()
        e_.synchronize()
        ms = s_.elapsed_time(e_) / iters
        out[name] = {"ms": round(ms, 4), "gbps": round(nbytes * 8 / ms / 1e6, 1)}
    del dst
    torch.cuda.empty_cache()
    return {"workload": f"AES-{keybits}, {nbytes // MIB} MiB", **out}


def run_stress(torch, aesgb, dev, total=16 * GIB, region=64 * MIB, iters=3):
    """Stress workload: AES-256 ECB decryption in place over 16 GiB of 64 MiB
    regions cycling uniform random / all-zero / one 16-byte block repeated.
    Timed as one launch per pass; afterwards every all-zero and periodic region
    must hold one repeated block (ECB's identical-block invariant), checked on
    the device."""
    import numpy as np
    from paper_1902_05234_gb300 import workloads as wl
    kinds = wl.stress_region_kinds(total, region)
    buf = torch.empty(total, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 110)
    hg = wl.rng(110)
    for r, kind in enumerate(kinds.tolist()):
        sl = buf[r * region:(r + 1) * region]
        if kind == 0:
            sl.random_(0, 256, generator=g)
        elif kind == 1:
            sl.zero_()
        else:
            blk = torch.from_numpy(hg.integers(0, 256, 16, dtype=np.uint8)).to(dev)
            sl.view(-1, 16).copy_(blk.expand(region // 16, 16))
    _, dec, nr = aesgb.aes_expand_key(256, wl.random_key(256, 110).tobytes())
    n = total // 16
    aesgb.aes_ecb_decrypt(dec, nr, buf, buf, n)            # warm-up pass (also in place)
    torch.cuda.synchronize()
    s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_.record()
    for _ in range(iters):
        aesgb.aes_ecb_decrypt(dec, nr, buf, buf, n)
    e_.record()
    e_.synchronize()
    ms = s_.elapsed_time(e_) / iters
    ok = True
    for r, kind in enumerate(kinds.tolist()):
        if kind:
            blocks = buf[r * region:(r + 1) * region].view(-1, 16)
            ok = ok and bool((blocks == blocks[0]).all())
    del buf
    torch.cuda.empty_cache()
    return {"workload": "AES-256 ECB decrypt in place, 16 GiB of 64 MiB regions: uniform / all-zero / "
                        "16-byte periodic", "ms": round(ms, 3), "gbps": round(total * 8 / ms / 1e6, 1),
            "identical_block_invariant": ok,
            "cfg": repr(aesgb.aes_ecb_get_cfg(1, nr, n))}


def run_gb300(args, dist: Dist):
    import torch
    from paper_1902_05234_gb300 import aesgb
    from paper_1902_05234_gb300 import workloads as wl

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    nbytes = args.bytes // 16 * 16
    nblocks = nbytes // 16
    key = wl.random_key(args.keybits, 30 + dist.rank).tobytes()

    pt = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 30 + dist.rank)
    pt.random_(0, 256, generator=g)
    ct = torch.empty_like(pt)
    back = torch.empty_like(pt)

    def step(ev=None, k=0):
        enc, dec, nr = aesgb.aes_expand_key(args.keybits, key)
        if ev is not None:
            ev[0][k].record(stream)
        aesgb.aes_ecb_encrypt(enc, nr, pt, ct, nblocks, stream)
        if ev is not None:
            ev[1][k].record(stream)
        aesgb.aes_ecb_decrypt(dec, nr, ct, back, nblocks, stream)
        if ev is not None:
            ev[2][k].record(stream)

    tuned = None
    if not args.no_tune:
        # the autotuner picks block size, bytes per thread and table layout for
        # this size, untimed; aes_ecb_encrypt/decrypt then use its choice
        enc0, dec0, nr0 = aesgb.aes_expand_key(args.keybits, key)
        tuned = {"enc": repr(aesgb.aes_tune_ecb(0, nr0, enc0, pt, ct, nblocks)),
                 "dec": repr(aesgb.aes_tune_ecb(1, nr0, dec0, pt, back, nblocks))}
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if not torch.equal(back, pt):
        raise SystemExit("bench: decrypt(encrypt(x)) != x")

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(K)] for _ in range(3)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(K):
        step(evs, k)
    t_end.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    enc_ms = statistics.mean(evs[0][k].elapsed_time(evs[1][k]) for k in range(K))
    dec_ms = statistics.mean(evs[1][k].elapsed_time(evs[2][k]) for k in range(K))
    if not torch.equal(back, pt):
        raise SystemExit("bench: decrypt(encrypt(x)) != x after the timed steps")

    world = dist.world
    ms_per_step, value = aggregate_throughput(dist, total_ms, 2 * nbytes * 8, K)
    clk = clocks.summary()

    # --- roofline of the encryption kernel --------------------------------
    nr = nrounds_of(args.keybits)
    sms = aesgb.aes_device_sm_count(dist.local)
    f_mhz = clk["sm_mhz"] or 2070.0
    lookup_bytes = nblocks * 16 * nr * 4                 # algorithmic smem lookup bytes per launch
    achieved_gbs = lookup_bytes / (enc_ms / 1e3) / 1e9
    peak_gbs = sms * f_mhz * 1e6 * 128 / 1e9             # 32 banks x 4 B per clock per SM
    peak_gbps_metric = sms * f_mhz * 1e6 * 256 / nr / 1e9
    enc_gbps = nbytes * 8 / enc_ms / 1e6
    dec_gbps = nbytes * 8 / dec_ms / 1e6
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # measured peak of the same bound: the lookup-rate calibration kernel
    sink = torch.empty(sms * 4096, dtype=torch.uint8, device=dev)
    cal_lookups, cal_s = aesgb.aes_calibrate_lookup_rate(sink, sink.numel(), stream)
    del sink
    measured_lookup_gbs = cal_lookups * 4 / cal_s / 1e9
    roofline = {
        "bound": "smem", "kernel": f"ecb_kernel<encrypt,Nr={nr}>",
        "achieved": round(achieved_gbs, 1), "peak": round(peak_gbs, 1), "unit": "GB/s",
        "frac": round(achieved_gbs / peak_gbs, 4),
        "traffic": recorded_traffic("ecb_encrypt", args.keybits, nbytes),
        "algorithmic_bytes_per_launch": lookup_bytes,
        "peak_basis": f"{sms} SMs x {f_mhz:.0f} MHz (median sampled under load) x 128 B/clk shared-memory "
                      f"lookups (derived from unit counts and the measured clock)",
        "achieved_gbps": round(enc_gbps, 1), "peak_gbps": round(peak_gbps_metric, 1),
        # the same data pipe also carries the 128-bit global loads and stores:
        # 64*Nr bytes of lookups + 32 bytes of I/O per block at 128 B/clk/SM
        "l1tex_bound_gbps": round(sms * f_mhz * 1e6 * 128 / (64 * nr + 32) * 128 / 1e9, 1),
        "l1tex_frac": round(enc_gbps / (sms * f_mhz * 1e6 * 128 / (64 * nr + 32) * 128 / 1e9), 4),
        "measured_peak": {"gbs": round(measured_lookup_gbs, 1),
                          "lookups_per_clk_per_sm": round(cal_lookups / cal_s / (sms * f_mhz * 1e6), 3),
                          "frac": round(achieved_gbs / measured_lookup_gbs, 4),
                          "source": "aes_calibrate_lookup_rate (conflict-free LDS stream, same table layout)"},
        "avg_launch_ms": round(enc_ms, 4),
        "hbm": {"achieved_gbs": round(2 * nbytes / (enc_ms / 1e3) / 1e9, 1), "peak_gbs": hbm_peak,
                "frac": round(2 * nbytes / (enc_ms / 1e3) / 1e9 / hbm_peak, 4), "peak_source": "measured"},
        "decrypt": {"avg_launch_ms": round(dec_ms, 4), "gbps": round(dec_gbps, 1),
                    "frac": round(lookup_bytes / (dec_ms / 1e3) / 1e9 / peak_gbs, 4)},
    }

    # --- end to end through the host-buffer entry point --------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, aesgb, key, args.keybits, pt, nbytes, stream, dist, K)

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args, world),
            "enc_gbps": round(enc_gbps, 1), "dec_gbps": round(dec_gbps, 1),
            "roofline": roofline, "e2e": e2e, "gpu_launches": 2 * K * world,
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} | {"samples": clk["samples"]},
            "launch_cfg": {"enc": repr(aesgb.aes_ecb_get_cfg(0, nr, nblocks)),
                           "dec": repr(aesgb.aes_ecb_get_cfg(1, nr, nblocks)), "tuned": tuned is not None}}
    del ct, back
    torch.cuda.empty_cache()
    if dist.rank == 0 and world == 1 and not args.no_sweep:
        line["sweep"] = run_sweep(torch, aesgb, dev, tune=not args.no_tune)
    if dist.rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = run_batched(torch, aesgb, dev, n=args.batch_n, tune=not args.no_tune,
                                      hi=args.batch_max_bytes)
        line["batched"]["roofline"] = batch_roofline(line["batched"], args.batch_n, args.batch_max_bytes,
                                                     sms, f_mhz)
    if dist.rank == 0 and world == 1:
        line["modes"] = run_modes(torch, aesgb, pt, nbytes, key, args.keybits)
    if dist.rank == 0 and world == 1 and not args.no_ct:
        line["constant_time"] = run_constant_time(torch, aesgb, pt, nbytes, key, args.keybits)
        sink = torch.empty(sms * 4096, dtype=torch.uint8, device=dev)
        logic_cal = aesgb.aes_calibrate_logic_rate(sink, sink.numel(), stream)
        del sink
        line["constant_time"]["roofline"] = ct_roofline(aesgb, line["constant_time"], nbytes, args.keybits,
                                                        sms, f_mhz, logic_cal)
    if dist.rank == 0 and world == 1 and not args.no_stress:
        line["stress"] = run_stress(torch, aesgb, dev)
    if dist.rank == 0 and world == 1 and not args.no_served:
        line["served"] = run_served(torch, aesgb, dev, n_req=args.served_requests, slots=args.served_slots)
    if dist.rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.keybits)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(torch, aesgb, key, keybits, pt_dev, nbytes, stream, dist, K):
    """Host plaintext -> encrypt -> host ciphertext -> decrypt -> host plaintext,
    all through aes_ecb_host with page-locked host buffers."""
    nblocks = nbytes // 16
    h_pt = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_ct = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_back = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_pt.copy_(pt_dev)

    def e2e_step():
        enc, dec, nr = aesgb.aes_expand_key(keybits, key)
        aesgb.aes_ecb_host_direct(0, enc, nr, h_pt, h_ct, nblocks, stream)
        aesgb.aes_ecb_host_direct(1, dec, nr, h_ct, h_back, nblocks, stream)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    iters = max(3, min(K, 10))
    dist.barrier()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(iters):
        e2e_step()
    e.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = dist.max(s.elapsed_time(e)) / iters
    if not torch.equal(h_back, h_pt):
        raise SystemExit("bench e2e: decrypt(encrypt(x)) != x")
    # the same steps through the staged pipeline (explicit copies on three streams)
    stage_bytes = 3 * 64 * MIB
    stage = torch.empty(stage_bytes, dtype=torch.uint8, device=pt_dev.device)
    h_back.zero_()

    def staged_step():
        enc, dec, nr = aesgb.aes_expand_key(keybits, key)
        aesgb.aes_ecb_host(0, enc, nr, h_pt, h_ct, nblocks, stage, stage_bytes, stream)
        aesgb.aes_ecb_host(1, dec, nr, h_ct, h_back, nblocks, stage, stage_bytes, stream)

    staged_step()
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(iters):
        staged_step()
    e.record(stream)
    torch.cuda.synchronize()
    ms_staged = dist.max(s.elapsed_time(e)) / iters
    if not torch.equal(h_back, h_pt):
        raise SystemExit("bench e2e (staged): decrypt(encrypt(x)) != x")
    del stage
    return {"value": round(2 * nbytes * 8 * dist.world / ms / 1e6, 2), "unit": UNIT,
            "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
            "ms_per_step": round(ms, 4),
            "api": "aes_ecb_host_direct (kernel reads/writes page-locked host memory over NVLink-C2C)",
            "steps": iters,
            "staged": {"value": round(2 * nbytes * 8 * dist.world / ms_staged / 1e6, 2), "ms_per_step": round(ms_staged, 4),
                       "api": "aes_ecb_host (cudaMemcpyAsync in/out through 3 x 64 MiB device slots)"}}


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.study:
            run_study(args)
        else:
            run_gb300(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
