"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no AES arithmetic: it only draws bytes, keys, message sizes,
directions and arrival times from seeded numpy generators (PCG64), so that the
GPU path and the CPU oracle are fed identical inputs.  The paper's own input
files are unspecified (section 5), so uniform random bytes stand in for them.

Workloads (sizes as used by the tests and the benchmark):

* ``ecb_1mib``      1 MiB = 65,536 blocks, one random 128-bit key.
* ``sweep``         single buffers of 1 MiB ... 4 GiB (powers of 4), AES-128/192/256.
* ``batch``         4,096 messages, lengths log-uniform 16 B .. 16 MiB (multiples of
                    16), per-message key size uniform over {128, 192, 256}, direction
                    50/50.
* ``served``        Poisson request stream, sizes log-uniform 64 B .. 4 MiB, keys drawn
                    from 1,024 resident schedules, direction 50/50.
* ``stress``        16 GiB in 64 MiB regions cycling uniform random / all-zero /
                    16-byte periodic.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 190205230
MIB = 1 << 20
GIB = 1 << 30


def rng(seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + int(seed_offset)))


def random_bytes(nbytes: int, seed_offset: int = 0) -> np.ndarray:
    """``nbytes`` uniform random bytes (uint8)."""
    return rng(seed_offset).integers(0, 256, size=int(nbytes), dtype=np.uint8)


def random_key(keybits: int, seed_offset: int = 0) -> np.ndarray:
    if keybits not in (128, 192, 256):
        raise ValueError(keybits)
    return rng(10_000 + seed_offset).integers(0, 256, size=keybits // 8, dtype=np.uint8)


def log_uniform_lengths(n: int, lo: int, hi: int, g: np.random.Generator) -> np.ndarray:
    """n lengths, log-uniform on [lo, hi], rounded down to multiples of 16 (>= 16)."""
    u = g.uniform(math.log(lo), math.log(hi), size=n)
    return (16 * np.maximum(1, np.floor(np.exp(u) / 16))).astype(np.int64)


def batch_workload(n: int = 4096, lo: int = 16, hi: int = 16 * MIB, seed_offset: int = 3):
    """Lengths (bytes), key sizes (bits) and directions (0 enc, 1 dec) of a batch."""
    g = rng(seed_offset)
    lengths = log_uniform_lengths(n, lo, hi, g)
    keybits = g.choice(np.array([128, 192, 256]), size=n)
    dirs = g.integers(0, 2, size=n)
    return lengths, keybits.astype(np.int64), dirs.astype(np.int64)


def served_workload(n_req: int, rate_per_s: float, n_keys: int = 1024, lo: int = 64,
                    hi: int = 4 * MIB, seed_offset: int = 4):
    """Poisson arrivals (seconds from start), sizes, key ids and directions."""
    g = rng(seed_offset)
    gaps = g.exponential(1.0 / rate_per_s, size=n_req)
    arrivals = np.cumsum(gaps)
    sizes = log_uniform_lengths(n_req, lo, hi, g)
    key_ids = g.integers(0, n_keys, size=n_req)
    dirs = g.integers(0, 2, size=n_req)
    return arrivals, sizes, key_ids.astype(np.int64), dirs.astype(np.int64)


def stress_region_kinds(total_bytes: int, region_bytes: int = 64 * MIB):
    """Kind of each region: 0 uniform random, 1 all-zero, 2 16-byte periodic."""
    nreg = (int(total_bytes) + region_bytes - 1) // region_bytes
    return np.arange(nreg, dtype=np.int64) % 3
