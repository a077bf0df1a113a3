"""Seeded synthetic workloads: shapes, seeds and sampled indices only.

This module holds none of the generators' arithmetic.  Both the CUDA-path
tests/bench and the oracle-side checks take their inputs from here, so the two
sides see identical problems.  The paper's workloads are the generators'
own output streams (no dataset is involved); the configurations below fix
the seeds, stream counts, lengths and mixes used for parity and timing.
"""
from __future__ import annotations

import numpy as np

# Generators of the bulk-fill configuration (64-bit: +, ++, ** on xoshiro256
# and xoroshiro128; 32-bit: ++ and ** on xoshiro128).
BULK_VARIANTS = (
    "xoshiro256+", "xoshiro256++", "xoshiro256**",
    "xoroshiro128+", "xoroshiro128++", "xoroshiro128**",
    "xoshiro128**", "xoshiro128++",
)
# The other generators of the paper's Sec. 5 (Tables 4, 5, 7, 8).
EXTRA_VARIANTS = ("xoroshiro128*", "xoroshiro64*", "xoroshiro64**", "xoshiro512+", "xoshiro512++",
                  "xoshiro512**", "xoroshiro1024*", "xoroshiro1024++", "xoroshiro1024**")
ALL_VARIANTS = BULK_VARIANTS + ("xoshiro128+",) + EXTRA_VARIANTS
# Generators whose states fit the 32-byte slots of batches and servers.
SLOT_VARIANTS = BULK_VARIANTS + ("xoshiro128+", "xoroshiro128*", "xoroshiro64*", "xoroshiro64**")

# xoshiro256**, SplitMix64(0x0123456789ABCDEF), 1024 streams by successive
# jumps, 1024 outputs each, as raw uint64 and as doubles.
CONFIG_PLAIN = dict(variant="xoshiro256**", seed=0x0123456789ABCDEF, kind="jump", S=1024, m=1024,
                    dtypes=("u64", "f64"))

# Bulk fill: every generator, SplitMix64(42) base, 2^20 streams by jumps,
# 2^10 outputs each (2^30 values), native words and doubles.
CONFIG_BULK = dict(variants=BULK_VARIANTS, seed=42, kind="jump", S=1 << 20, m=1 << 10)

# Jump-start at scale: 2^24 xoshiro256++ streams J^i(s0) and L^i(s0), 64
# outputs each; 4096 uniformly sampled stream indices (seed 1) are checked.
CONFIG_JUMPSTART = dict(variant="xoshiro256++", seed=42, kinds=("jump", "long"), S=1 << 24, m=64,
                        samples=4096, sample_seed=1)


def native_dtype(variant: str) -> str:
    return "u32" if variant.startswith(("xoshiro128", "xoroshiro64")) else "u64"


def sample_indices(S: int, count: int, seed: int) -> np.ndarray:
    """count sorted distinct stream indices in [0, S): 0 and S-1 plus
    count - 2 uniform draws without replacement from the indices between."""
    rng = np.random.default_rng(seed)
    if count >= S:
        return np.arange(S, dtype=np.int64)
    inner = rng.choice(S - 2, size=max(count - 2, 0), replace=False) + 1 if count > 2 else np.zeros(0, np.int64)
    idx = np.concatenate([[0, S - 1], inner])[:count]
    return np.sort(idx.astype(np.int64))


# (S, m) shapes for element-by-element parity: single values, partial tiles,
# several 32-stream tiles and 128-byte rows, ragged tails in both dimensions.
PARITY_SHAPES = ((1, 1), (1, 15), (2, 17), (31, 16), (33, 33), (129, 100), (300, 64),
                 (257, 1000), (1000, 48))


def random_states(k: int, w: int, count: int, seed: int) -> np.ndarray:
    """count nonzero states of k words of w bits (uint64 array [count, k])."""
    rng = np.random.default_rng(seed)
    hi = np.uint64(2**w - 1) if w < 64 else np.uint64(2**64 - 1)
    out = rng.integers(0, hi, size=(count, k), dtype=np.uint64, endpoint=True)
    zero = ~out.any(axis=1)
    out[zero, 0] = 1
    return out


# Batched uneven requests: 4096 requests, request r seeded with SplitMix64(r),
# generator uniform over the 8 bulk generators, length log-uniform in
# [1, 2^24], output type uniform over {native word, double}.
CONFIG_BATCH = dict(nreq=4096, max_len=1 << 24, mix_seed=4)


def batch_requests(nreq=4096, max_len=1 << 24, mix_seed=4, variants=BULK_VARIANTS):
    """[(variant, dtype, n, seed)] for the batched configuration."""
    rng = np.random.default_rng(mix_seed)
    v = rng.integers(0, len(variants), size=nreq)
    dt = rng.integers(0, 2, size=nreq)
    n = np.floor(np.exp(rng.uniform(0.0, np.log(max_len + 1.0), size=nreq))).astype(np.int64)
    n = np.clip(n, 1, max_len)
    out = []
    for r in range(nreq):
        name = variants[int(v[r])]
        out.append((name, native_dtype(name) if dt[r] == 0 else "f64", int(n[r]), r))
    return out


# Serving: 256 clients (half xoshiro256**, half xoroshiro128++) with
# device-resident states seeded by SplitMix64(client), Poisson arrivals at
# 20k requests/s, sizes log-uniform in [2^10, 2^26] values, output type
# uniform over {uint64, double}, a 16 GiB output budget.
CONFIG_SERVE = dict(nclients=256, rate=20000.0, min_len=1 << 10, max_len=1 << 26, arena_bytes=16 << 30,
                    trace_seed=6)


def serve_clients(nclients=256):
    return [("xoshiro256**" if c % 2 == 0 else "xoroshiro128++") for c in range(nclients)], list(range(nclients))


def serve_trace(nreq, nclients=256, rate=20000.0, min_len=1 << 10, max_len=1 << 26, trace_seed=6, **_):
    """(arrival_us, client, n, dtype) arrays for nreq Poisson arrivals."""
    rng = np.random.default_rng(trace_seed)
    gaps = rng.exponential(1e6 / rate, size=nreq) if rate > 0 else np.zeros(nreq)
    arrival = np.cumsum(gaps) - gaps[0]
    client = rng.integers(0, nclients, size=nreq).astype(np.uint32)
    n = np.floor(np.exp(rng.uniform(np.log(min_len), np.log(max_len + 1.0), size=nreq))).astype(np.uint64)
    n = np.clip(n, min_len, max_len)
    dtype = np.where(rng.integers(0, 2, size=nreq) == 0, "u64", "f64")
    return arrival, client, n, list(dtype)


# Bulk linear complexity (Sec. 9.3): every output bit of the 8 bulk
# generators (64 or 32 bits each, 448 sequences), the first 2^16 outputs
# from SplitMix64(1).  Low bits of the + generators have the small
# complexities of Table 13; the others come out near N / 2.
CONFIG_LC_BULK = dict(variants=BULK_VARIANTS, N=1 << 16, seed=1)


def lc_bulk_jobs(variants=BULK_VARIANTS, N=1 << 16, **_):
    """[(variant, bit, N)] for the bulk linear-complexity configuration."""
    return [(v, b, N) for v in variants for b in range(32 if native_dtype(v) == "u32" else 64)]
