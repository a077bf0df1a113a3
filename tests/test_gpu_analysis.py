"""The paper's analysis workloads on the device, against the oracle and the
paper: escaping zeroland (Sec. 8) and the linear complexity of single output
bits by Berlekamp-Massey (Sec. 9.3, Table 13).  Integer results: bit-exact."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xr():
    from paper_1805_01407_gb300 import build
    build.build()
    import paper_1805_01407_gb300 as xr
    return xr


@pytest.fixture(scope="module")
def ctx(xr):
    c = xr.Context(0)
    yield c
    c.close()


# ------------------------------------------------------------------ zeroland

@pytest.mark.parametrize("name", W.ALL_VARIANTS)
def test_zeroland_equals_oracle(ctx, name):
    """The paper's setting: 1000 outputs, windows of 4."""
    got = ctx.zeroland(name, 1000, 4).cpu().numpy().astype(np.uint64)
    assert (got == O.zeroland(name, 1000, 4)).all()


@pytest.mark.parametrize("name,nout,window", [("xoshiro256**", 1, 1), ("xoroshiro128+", 64, 64),
                                              ("xoshiro128**", 5000, 1), ("xoroshiro64*", 300, 63),
                                              ("xoroshiro1024++", 130, 7), ("xoshiro512+", 2, 2)])
def test_zeroland_window_edges(ctx, name, nout, window):
    got = ctx.zeroland(name, nout, window).cpu().numpy().astype(np.uint64)
    assert (got == O.zeroland(name, nout, window)).all()


def test_zeroland_first_output_closed_form(ctx):
    """One bits of the first output over the one-bit states (derived by hand
    from the scramblers' definitions; the same numbers pin the oracle)."""
    want = {"xoroshiro128+": 128, "xoshiro256++": 192, "xoshiro256**": 246, "xoroshiro128**": 246,
            "xoshiro128**": 118, "xoshiro128++": 96}
    for name, v in want.items():
        assert int(ctx.zeroland(name, 3, 1)[0]) == v, name


def test_zeroland_rejects_bad_windows(ctx, xr):
    for nout, window in ((10, 0), (100, 65), (3, 4)):
        with pytest.raises(xr.XRError):
            ctx.zeroland("xoshiro256**", nout, window)


# ------------------------------------------------------------------ linear complexity

def seeded(ctx, name, seed):
    st = ctx.empty_states(name, 1)
    ctx.seed(name, seed, st)
    return st


def _table13(golden):
    rows = [(g, int(b), int(lc)) for g, b, lc in golden("plus_linear_complexity.txt")]
    return [r for r in rows if not r[0].startswith("engine/")]


def test_linear_complexity_table13(ctx, golden):
    """Every generator row of Table 13 (the lowest bits of the + generators),
    computed on the device from 2 L + 200 bits."""
    for g, b, lc in _table13(golden):
        assert ctx.linear_complexity(g, b, 2 * lc + 200, seeded(ctx, g, 1)) == lc, (g, b)


@pytest.mark.parametrize("name,bit,N", [("xoshiro256**", 63, 20000), ("xoshiro256++", 0, 6000),
                                        ("xoroshiro128**", 5, 9001), ("xoroshiro128++", 40, 4097),
                                        ("xoshiro128**", 31, 8000), ("xoroshiro64**", 3, 3333),
                                        ("xoshiro512**", 17, 5000), ("xoroshiro1024++", 62, 7000),
                                        ("xoroshiro128+", 3, 70000), ("xoroshiro128*", 60, 12345)])
def test_linear_complexity_equals_oracle(ctx, name, bit, N):
    """Nonlinear bits (complexity close to N / 2) and a Table 13 bit whose
    complexity exceeds what N bits decide."""
    for seed in (1, 99):
        assert ctx.linear_complexity(name, bit, N, seeded(ctx, name, seed)) == \
            O.linear_complexity(name, bit, N, seed), (name, bit, N, seed)


@pytest.mark.parametrize("name,bit,N", [("xoroshiro128+", 1, 200000), ("xoshiro256+", 0, 600001),
                                        ("xoroshiro128+", 1, 780000), ("xoshiro256+", 1, 786000)])
def test_linear_complexity_long_prefixes(ctx, xr, name, bit, N):
    """Long prefixes of low-complexity bits (4, 8 and 12 polynomial words per
    thread, up to the largest prefix accepted)."""
    assert N <= xr.XR_LC_MAX_BITS
    assert ctx.linear_complexity(name, bit, N, seeded(ctx, name, 7)) == O.linear_complexity(name, bit, N, 7)


@pytest.mark.parametrize("N", [2, 3, 31, 32, 33, 63, 64, 65, 127, 1000, 1025])
def test_linear_complexity_short_prefixes(ctx, N):
    for name, bit in (("xoshiro256+", 0), ("xoshiro256**", 40), ("xoshiro128++", 7)):
        assert ctx.linear_complexity(name, bit, N, seeded(ctx, name, 5)) == \
            O.linear_complexity(name, bit, N, 5), (name, bit, N)


def test_linear_complexity_leaves_the_state(ctx):
    st = seeded(ctx, "xoshiro256+", 3)
    before = st.clone()
    ctx.linear_complexity("xoshiro256+", 1, 1000, st)
    assert bool((st == before).all())


def test_linear_complexity_rejects_bad_args(ctx, xr):
    st = seeded(ctx, "xoshiro128+", 1)
    for bit, N in ((32, 100), (-1, 100), (0, 1), (0, xr.XR_LC_MAX_BITS + 1)):
        with pytest.raises(xr.XRError):
            ctx.linear_complexity("xoshiro128+", bit, N, st)


# ------------------------------------------------------------------ many at once

def states_for(ctx, xr, jobs, seeds):
    import torch
    st = torch.zeros(len(jobs) * 128, dtype=torch.uint8, device="cuda")
    for j, ((v, _, _), sd) in enumerate(zip(jobs, seeds)):
        ctx.seed(v, sd, st[j * 128:])
    return st


def test_linear_complexity_many_table13(ctx, xr, golden):
    """All generator rows of Table 13 in one call."""
    rows = _table13(golden)
    jobs = [(g, b, 2 * lc + 200) for g, b, lc in rows]
    got = ctx.linear_complexity_many(jobs, states_for(ctx, xr, jobs, [1] * len(jobs)))
    assert got == [lc for _, _, lc in rows]


def test_linear_complexity_many_equals_oracle(ctx, xr):
    """A mixed batch (every generator, low and high bits, prefixes from 2 to
    40000 bits, repeated jobs) against the oracle job by job, and against the
    single call."""
    rng = np.random.default_rng(11)
    jobs, seeds = [], []
    for j in range(60):
        v = W.ALL_VARIANTS[j % len(W.ALL_VARIANTS)]
        bit = int(rng.integers(0, O.word_bits(v)))
        N = int(np.exp(rng.uniform(np.log(2), np.log(40000))))
        jobs.append((v, bit, N))
        seeds.append(int(rng.integers(1, 1 << 40)))
    jobs += jobs[:3]
    seeds += seeds[:3]
    got = ctx.linear_complexity_many(jobs, states_for(ctx, xr, jobs, seeds))
    for (v, bit, N), sd, L in zip(jobs, seeds, got):
        assert L == O.linear_complexity(v, bit, N, sd), (v, bit, N, sd)
    for k in (0, 7, 31):
        v, bit, N = jobs[k]
        assert ctx.linear_complexity(v, bit, N, seeded(ctx, v, seeds[k])) == got[k]


def test_linear_complexity_many_rejects_a_bad_job(ctx, xr):
    import torch
    st = torch.zeros(3 * 128, dtype=torch.uint8, device="cuda")
    with pytest.raises(xr.XRError):
        ctx.linear_complexity_many([("xoshiro256+", 0, 100), ("xoshiro128+", 40, 100), ("xoshiro256+", 1, 100)], st)
    assert ctx.linear_complexity_many([], st) == []


def test_linear_complexity_bulk_configuration_full(ctx, xr):
    """The bulk configuration (every bit of the 8 bulk generators, 2^16 bits):
    all 448 sequences in one call, every one against the oracle's
    Berlekamp-Massey (run on every host core: the oracle's C calls release the
    GIL); bit 0 of the + generators has the complexity of Table 13 (n)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    c = W.CONFIG_LC_BULK
    jobs = W.lc_bulk_jobs(**c)
    got = ctx.linear_complexity_many(jobs, states_for(ctx, xr, jobs, [c["seed"]] * len(jobs)))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with ThreadPoolExecutor(cores) as ex:
        want = list(ex.map(lambda j: O.linear_complexity(j[0], j[1], j[2], c["seed"]), jobs))
    for k, job in enumerate(jobs):
        assert got[k] == want[k], job
    for k, (v, b, N) in enumerate(jobs):
        if b == 0 and v.endswith("+") and not v.endswith("++"):
            assert got[k] == O.state_bits(v), v
        assert got[k] is not None and 0 < got[k] <= N // 2 + 64


def _oracle_all(jobs, seeds):
    import os
    from concurrent.futures import ThreadPoolExecutor
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with ThreadPoolExecutor(cores) as ex:
        return list(ex.map(lambda a: O.linear_complexity(a[0][0], a[0][1], a[0][2], a[1]), zip(jobs, seeds)))


def test_linear_complexity_cluster_threshold(ctx, xr):
    """Calls of up to SMs / 8 sequences run each sequence on a cluster of 8
    CTAs, larger calls one CTA per sequence: the same mixed jobs (lengths from
    300 to 60000 bits, low and high bits, every engine size) at the threshold
    and one above it, against the oracle, and the first jobs against the
    single call (which also takes the cluster path)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    k = sms // 8
    rng = np.random.default_rng(23)
    jobs, seeds = [], []
    for j in range(k + 1):
        v = W.ALL_VARIANTS[(3 * j) % len(W.ALL_VARIANTS)]
        jobs.append((v, int(rng.integers(0, O.word_bits(v))), int(np.exp(rng.uniform(np.log(300), np.log(60000))))))
        seeds.append(int(rng.integers(1, 1 << 40)))
    want = _oracle_all(jobs, seeds)
    for m in (k, k + 1):
        got = ctx.linear_complexity_many(jobs[:m], states_for(ctx, xr, jobs[:m], seeds[:m]))
        assert got == want[:m], m
    for j in range(3):
        v, bit, N = jobs[j]
        assert ctx.linear_complexity(v, bit, N, seeded(ctx, v, seeds[j])) == want[j]


@pytest.mark.parametrize("name,count,Nmax", [("xoshiro256**", 40, 70000), ("xoroshiro1024++", 33, 20000)])
def test_linear_complexity_many_long_run_of_one_generator(ctx, xr, name, count, Nmax):
    """A run of at least 32 sequences of one generator takes the bit kernel
    with one sequence per lane: lengths from 2 to Nmax in one run (sequences
    that end in different chunks, and in the first), with and without the
    engine's power sets (xoroshiro1024 jumps with its T^(2^k) tables)."""
    rng = np.random.default_rng(count)
    jobs, seeds = [], []
    for j in range(count):
        N = 2 if j == 0 else (Nmax if j == 1 else int(np.exp(rng.uniform(np.log(2), np.log(Nmax)))))
        jobs.append((name, int(rng.integers(0, O.word_bits(name))), N))
        seeds.append(int(rng.integers(1, 1 << 40)))
    got = ctx.linear_complexity_many(jobs, states_for(ctx, xr, jobs, seeds))
    assert got == _oracle_all(jobs, seeds)


def test_linear_complexity_one_cta_long_sequences(ctx, xr):
    """Calls of more than SMs / 8 sequences run one CTA per sequence; long
    ones there take 8 words per thread (up to 8192 words) or 12 (beyond):
    three sequences of 600,000 to 786,000 bits and two of 300,000 and
    400,000 among short ones, against the oracle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = sms // 8 + 1
    long_ = [("xoroshiro128+", 1, 600001), ("xoshiro256+", 1, 700000), ("xoroshiro128+", 2, 786000),
             ("xoshiro256**", 30, 300000), ("xoroshiro128++", 5, 400000)]
    rng = np.random.default_rng(31)
    jobs = list(long_)
    while len(jobs) < count:
        v = W.ALL_VARIANTS[len(jobs) % len(W.ALL_VARIANTS)]
        jobs.append((v, int(rng.integers(0, O.word_bits(v))), int(rng.integers(2, 5000))))
    seeds = [int(rng.integers(1, 1 << 40)) for _ in jobs]
    got = ctx.linear_complexity_many(jobs, states_for(ctx, xr, jobs, seeds))
    assert got == _oracle_all(jobs, seeds)


@pytest.mark.parametrize("N", [64 * (2048 - 5), 64 * (2049 - 5)])
def test_linear_complexity_cluster_words_per_thread_boundary(ctx, N):
    """Single calls (cluster kernel) on both sides of its change from 2 to 4
    words per thread (2048 polynomial words)."""
    for name, bit in (("xoshiro256**", 11), ("xoroshiro128+", 0)):
        assert ctx.linear_complexity(name, bit, N, seeded(ctx, name, 4)) == O.linear_complexity(name, bit, N, 4)
