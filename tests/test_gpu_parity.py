"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every integer result is compared bit for bit; doubles and floats are compared
as bit patterns too (the conversions are exact, Sec. 5.3, so the tolerance is
zero).  Small shapes cover single values, partial tiles and ragged tails;
the plain, bulk and jump-start configurations are compared in full.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from xr_testutil import (assert_bits_equal, dense_from_library_columns, dense_from_oracle_rows,
                         expected, out_to_numpy, states_from_device, states_to_bytes,
                         states_to_device)

pytestmark = pytest.mark.gpu

GUARD = 64          # canary elements on each side of an output buffer
CANARY = 0x5A


@pytest.fixture(scope="module")
def xr():
    from paper_1805_01407_gb300 import build
    build.build()
    import paper_1805_01407_gb300 as xr
    return xr


@pytest.fixture(scope="module")
def ctx(xr):
    import torch
    assert torch.cuda.is_available()
    c = xr.Context(0)
    yield c
    c.close()


def guarded_output(xr, n, dtype, offset=0):
    """Output view of n elements with canary bytes on both sides."""
    import torch
    es = xr.dtype_bytes(dtype)
    total = (n + 2 * GUARD) * es + offset
    raw = torch.full((total,), CANARY, dtype=torch.uint8, device="cuda")
    start = GUARD * es + offset
    view = raw[start:start + n * es]
    return raw, view, start, n * es


def check_canaries(raw, start, nbytes):
    r = raw.cpu().numpy()
    assert (r[:start] == CANARY).all(), "write before the output"
    assert (r[start + nbytes:] == CANARY).all(), "write past the output"


def as_dtype(view, dtype):
    import torch
    tdt = {"u64": torch.int64, "u32": torch.int32, "f64": torch.float64, "f32": torch.float32}[dtype]
    return view.view(tdt)


# ------------------------------------------------------------------ tables

@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128+", "xoroshiro128++", "xoshiro128++",
                                  "xoroshiro64*", "xoshiro512+", "xoroshiro1024++"])
def test_jump_tables_match_oracle(ctx, xr, name):
    """T built on the device by stepping unit states equals the oracle's T (which
    equals the paper's block matrix); the squaring chain gives T^2, T^(2^d) and
    wraps around (T^(2^n) = T)."""
    n = O.state_bits(name)
    T = O.matrix_from_step(name)
    assert (dense_from_library_columns(ctx.jump_table(name, 0), n) == dense_from_oracle_rows(T)).all()
    T2 = O.mat_mul(T, T)
    assert (dense_from_library_columns(ctx.jump_table(name, 1), n) == dense_from_oracle_rows(T2)).all()
    if n > 256:
        return  # squaring the large matrices hundreds of times on the CPU takes too long
    d = xr.jump_log2(name, "jump")
    Td = O.mat_pow2(T, d)
    assert (dense_from_library_columns(ctx.jump_table(name, d), n) == dense_from_oracle_rows(Td)).all()
    last = dense_from_library_columns(ctx.jump_table(name, n - 1), n)
    sq = (last.astype(np.int64) @ last.astype(np.int64)) % 2
    assert (sq == dense_from_oracle_rows(T)).all()


# ------------------------------------------------------------------ seeding

@pytest.mark.parametrize("name", W.ALL_VARIANTS)
def test_seed(ctx, xr, name):
    import torch
    for seed in (0, 1, 42, 0x0123456789ABCDEF, 2**64 - 1):
        st = ctx.empty_states(name, 1)
        ctx.seed(name, seed, st)
        torch.cuda.synchronize()
        assert (states_from_device(name, st)[0] == O.seed(name, seed)).all()
        assert ctx.get_state(name, st) == states_to_bytes(name, O.seed(name, seed))


def test_seed_many(ctx, xr):
    import torch
    seeds = torch.arange(4096, dtype=torch.int64, device="cuda")
    for name in ("xoshiro256++", "xoroshiro128**", "xoshiro128**"):
        st = ctx.empty_states(name, 4096)
        ctx.seed_many(name, seeds, st)
        got = states_from_device(name, st)
        for s in (0, 1, 17, 4095):
            assert (got[s] == O.seed(name, s)).all()
        want = np.stack([O.seed(name, s) for s in range(4096)])
        assert (got == want).all()


# ------------------------------------------------------------------ fill

@pytest.mark.parametrize("name", W.ALL_VARIANTS)
@pytest.mark.parametrize("layout", ["stream", "interleaved"])
def test_fill_small_shapes(ctx, xr, name, layout):
    """All dtypes and shapes with ragged tails, canaries, write-back."""
    import torch
    w = O.word_bits(name)
    for si, (S, m) in enumerate(W.PARITY_SHAPES):
        starts = W.random_states(O.state_words(name), w, S, seed=1000 + si)
        raw = O.fill_streams(name, starts, m).reshape(S, m)
        for dtype in (xr.native_dtype(name), "f64", "f32"):
            d_states = states_to_device(name, starts)
            buf, view, start, nb = guarded_output(xr, S * m, dtype)
            ctx.fill(name, d_states, S, m, dtype, as_dtype(view, dtype), layout=layout, write_back=True)
            torch.cuda.synchronize()
            check_canaries(buf, start, nb)
            got = out_to_numpy(as_dtype(view, dtype), dtype).reshape((S, m) if layout == "stream" else (m, S))
            if layout == "interleaved":
                got = got.T
            want = expected(name, raw.reshape(-1), dtype).reshape(S, m)
            assert_bits_equal(got.reshape(-1), want.reshape(-1), "%s %s S=%d m=%d" % (name, dtype, S, m))
            after = states_from_device(name, d_states)
            for i in (0, S // 2, S - 1):
                assert (after[i] == O.step(name, starts[i], m)).all()
    assert ctx.status() == 0


@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128++", "xoshiro128**"])
def test_fill_unaligned_output_and_no_write_back(ctx, xr, name):
    """An output pointer that is element- but not 16-byte aligned takes the
    plain-store path; without write-back the states are unchanged."""
    import torch
    S, m = 77, 40
    starts = W.random_states(O.state_words(name), O.word_bits(name), S, seed=7)
    raw = O.fill_streams(name, starts, m)
    for dtype in (xr.native_dtype(name), "f64"):
        es = xr.dtype_bytes(dtype)
        d_states = states_to_device(name, starts)
        buf, view, start, nb = guarded_output(xr, S * m, dtype, offset=es)
        ctx.fill(name, d_states, S, m, dtype, as_dtype(view, dtype))
        torch.cuda.synchronize()
        check_canaries(buf, start, nb)
        assert_bits_equal(out_to_numpy(as_dtype(view, dtype), dtype), expected(name, raw, dtype))
        assert (states_from_device(name, d_states) == starts).all()


def test_fill_continues_across_calls(ctx, xr):
    """Write-back makes two fills of m outputs equal one fill of 2m."""
    import torch
    name = "xoshiro256++"
    S, m = 500, 48
    starts = W.random_states(4, 64, S, seed=9)
    d_states = states_to_device(name, starts)
    a = ctx.empty_output(S * m, "u64")
    b = ctx.empty_output(S * m, "u64")
    ctx.fill(name, d_states, S, m, "u64", a, write_back=True)
    ctx.fill(name, d_states, S, m, "u64", b, write_back=True)
    torch.cuda.synchronize()
    raw = O.fill_streams(name, starts, 2 * m).reshape(S, 2 * m)
    assert_bits_equal(out_to_numpy(a, "u64").reshape(S, m), raw[:, :m])
    assert_bits_equal(out_to_numpy(b, "u64").reshape(S, m), raw[:, m:])


@pytest.mark.parametrize("name,w", [("xoshiro256+", 64), ("xoroshiro128+", 64), ("xoshiro128+", 32)])
def test_conversion_edge_values(ctx, xr, name, w):
    """Crafted + states whose first output is an edge value of the double and
    float conversions (0, values below 2^11, around 2^32, the top of the range):
    the + output is s_p + s_q, so (x, ..., 0) emits x first."""
    import torch
    k = O.state_words(name)
    X = [0, 1, 2**11 - 1, 2**11, 2**12 + 5, 2**24 - 1, 2**31, 2**32 - 1]
    if w == 64:
        X += [2**32, 2**32 + 2**31, 2**43 + 1, 2**53, 2**63, 2**64 - 1, 2**64 - 2**11]
    starts = []
    for x in X:
        if k == 2:          # xoroshiro128+: s0 + s1
            starts.append([x, 0] if x else [2**63, 2**63])
        else:               # xoshiro: s0 + s3
            starts.append([x, 0x1234567, 0x89ABCDE, 0])
    starts = np.array(starts, dtype=np.uint64)
    raw = O.fill_streams(name, starts, 16)
    assert [int(v) for v in raw.reshape(len(X), 16)[:, 0]] == X
    for dtype in ("f64", "f32", xr.native_dtype(name)):
        d_states = states_to_device(name, starts)
        out = ctx.empty_output(len(X) * 16, dtype)
        ctx.fill(name, d_states, len(X), 16, dtype, out)
        torch.cuda.synchronize()
        assert_bits_equal(out_to_numpy(out, dtype), expected(name, raw, dtype), dtype)


# ------------------------------------------------------------------ jumps

@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoroshiro128++", "xoshiro128++",
                                  "xoroshiro64**", "xoshiro512**", "xoroshiro1024*"])
def test_jump_and_advance(ctx, xr, name):
    import torch
    k, w = O.state_words(name), O.word_bits(name)
    states = W.random_states(k, w, 100, seed=11)
    for kind in ("jump", "long"):
        d = O.jump_log2(name, kind)
        for times in (1, 2, 5, 2**33 + 1):
            t = states_to_device(name, states)
            ctx.jump(name, kind, t, 100, times)
            got = states_from_device(name, t)
            for i in (0, 1, 50, 99):
                assert (got[i] == O.jump_pow(name, d, times, states[i])).all(), (kind, times, i)
    for nsteps in (1, 3, 1000, 2**40 + 12345):
        t = states_to_device(name, states)
        ctx.advance(name, t, 100, nsteps)
        got = states_from_device(name, t)
        for i in (0, 42, 99):
            want = O.step(name, states[i], nsteps) if nsteps <= 1000 else O.jump_pow(name, 0, nsteps, states[i])
            assert (got[i] == want).all(), (nsteps, i)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoroshiro128++", "xoshiro128**",
                                  "xoroshiro64*", "xoshiro512++", "xoroshiro1024++"])
@pytest.mark.parametrize("kind", ["jump", "long"])
def test_make_streams(ctx, xr, name, kind):
    """Stream i = J^(first + i)(base), against one jump after another."""
    base = O.seed(name, 42)
    d_base = states_to_device(name, base[None, :])
    for S, first in ((1, 0), (2, 0), (3, 5), (257, 0), (512, 0), (513, 3), (1000, 1), (3000, 777),
                     (600, 2**40 + 5)):
        out = ctx.empty_states(name, S)
        ctx.make_streams(name, kind, d_base, first, S, out)
        got = states_from_device(name, out)
        want = O.streams(name, kind, base, S, first=first)
        assert (got == want).all(), (S, first)


@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoroshiro128++", "xoshiro128**", "xoroshiro64*"])
@pytest.mark.parametrize("kind", ["jump", "long"])
def test_make_streams_chunked(ctx, xr, name, kind):
    """From 512 x 32 streams on, a chunk of 512 P streams takes its streams
    p + P j from one launch over the power set of the distance 2^J P; the rest
    of the range follows.  One chunk (P = 32); a chunk and a rest below it;
    two chunks (P = 64, then 32) and a rest, from a nonzero first; a chunk
    ending at stream 2^64 - 1: every state against one jump after another."""
    base = O.seed(name, 5)
    d_base = states_to_device(name, base[None, :])
    for S, first in ((16384, 0), (16384 + 77, 3), (3 * 16384 + 5, 1000), (16384, 2**64 - 16384)):
        out = ctx.empty_states(name, S)
        ctx.make_streams(name, kind, d_base, first, S, out)
        got = states_from_device(name, out)
        want = O.streams(name, kind, base, S, first=first)
        assert (got == want).all(), (S, first, int(np.argmax((got != want).any(axis=1))))
    assert ctx.status() == 0


@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128++"])
def test_make_streams_three_levels_sampled(ctx, xr, name):
    """More than 2^18 streams use all three levels of the start-state scheme;
    sampled indices around every level boundary against the oracle."""
    base = O.seed(name, 99)
    d_base = states_to_device(name, base[None, :])
    S, first = (1 << 18) + 1000, 12345
    out = ctx.empty_states(name, S)
    ctx.make_streams(name, "jump", d_base, first, S, out)
    got = states_from_device(name, out)
    d = O.jump_log2(name, "jump")
    idx = sorted(set([0, 1, 511, 512, 513, 1023, 1024, 262143, 262144, 262145, S - 1]) |
                 set(int(i) for i in W.sample_indices(S, 40, seed=4)))
    for i in idx:
        assert (got[i] == O.jump_pow(name, d, first + i, base)).all(), i


def test_make_streams_rejects_overlap(ctx, xr):
    name = "xoshiro256**"
    t = ctx.empty_states(name, 10)
    ctx.seed(name, 1, t)
    with pytest.raises(xr.XRError):
        ctx.make_streams(name, "jump", t, 0, 10, t)


# ------------------------------------------------------------------ one long sequence

@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128+", "xoroshiro128++", "xoshiro128++",
                                  "xoroshiro128*", "xoroshiro64**", "xoshiro512+", "xoroshiro1024**"])
def test_fill_seq(ctx, xr, name):
    import torch
    s0 = O.seed(name, 123)
    for n in (1, 2, 17, 1023, 1024, 1025, 4096, 70001):
        raw, after = O.generate(name, s0, n)
        for dtype in (xr.native_dtype(name), "f64"):
            d_state = states_to_device(name, s0[None, :])
            buf, view, start, nb = guarded_output(xr, n, dtype)
            ctx.fill_seq(name, d_state, n, dtype, as_dtype(view, dtype))
            torch.cuda.synchronize()
            check_canaries(buf, start, nb)
            assert_bits_equal(out_to_numpy(as_dtype(view, dtype), dtype), expected(name, raw, dtype),
                              "%s n=%d" % (name, n))
            assert (states_from_device(name, d_state)[0] == after).all()


@pytest.mark.parametrize("name,dtype", [("xoshiro256**", "u64"), ("xoroshiro128++", "f64"), ("xoshiro128+", "u32")])
def test_fill_seq_long_full(ctx, xr, name, dtype):
    """One sequence of 2^28 + 5000 values (2^18 + 5 segments of 2^10, so the
    segment starts use all three power-set levels and a ragged tail), with
    canaries, every value against the oracle: chunks of 2^20 values started
    by the oracle's own jump polynomial (x^(k 2^20) mod p), on every host core;
    and the state advanced by n."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    n, chunk = (1 << 28) + 5000, 1 << 20
    s0 = O.seed(name, 4242)
    d_state = states_to_device(name, s0[None, :])
    buf, view, start, nb = guarded_output(xr, n, dtype)
    ctx.fill_seq(name, d_state, n, dtype, as_dtype(view, dtype))
    torch.cuda.synchronize()
    check_canaries(buf, start, nb)
    got = out_to_numpy(as_dtype(view, dtype), dtype)
    assert (states_from_device(name, d_state)[0] == O.jump_pow(name, 0, n, s0)).all()

    def work(k0):
        cnt = min(chunk, n - k0)
        raw, _ = O.generate(name, O.jump_pow(name, 0, k0, s0) if k0 else s0, cnt)
        assert_bits_equal(got[k0:k0 + cnt], expected(name, raw, dtype), "%s values %d.." % (name, k0))
        return cnt

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with ThreadPoolExecutor(cores) as ex:
        assert sum(ex.map(work, range(0, n, chunk))) == n
    assert ctx.status() == 0


# ------------------------------------------------------------------ configurations

def test_plain_configuration_full(ctx, xr):
    """xoshiro256**, SplitMix64(0x0123456789ABCDEF), 1024 streams made by 1023
    successive jumps, 1024 outputs each: every value, as uint64 and double."""
    import torch
    c = W.CONFIG_PLAIN
    name, S, m = c["variant"], c["S"], c["m"]
    base = O.seed(name, c["seed"])
    starts = O.streams(name, "jump", base, S)          # one jump after another
    raw = O.fill_streams(name, starts, m)
    d_base = ctx.empty_states(name, 1)
    ctx.seed(name, c["seed"], d_base)
    d_states = ctx.empty_states(name, S)
    ctx.make_streams(name, "jump", d_base, 0, S, d_states)
    assert (states_from_device(name, d_states) == starts).all()
    for dtype in c["dtypes"]:
        out = ctx.empty_output(S * m, dtype)
        ctx.fill(name, d_states, S, m, dtype, out)
        torch.cuda.synchronize()
        assert_bits_equal(out_to_numpy(out, dtype), expected(name, raw, dtype), dtype)
        if dtype == "f64":
            v = out_to_numpy(out, dtype)
            assert v.min() >= 0.0 and v.max() < 1.0
            assert_bits_equal(v, (raw >> np.uint64(11)).astype(np.float64) * 2.0**-53)


def _host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def compare_streams_in_full(name, kind, base, S, m, d_states, outs, slice_streams=1 << 12):
    """Every start state (unless d_states is None) and every output of S
    streams J^i(base), i < S, against the oracle.  The device results are
    copied back slice by slice (slice_streams streams each) by this thread;
    the oracle computes the matching slices on every host core (worker
    threads: the oracle's C calls run without the GIL), one single-threaded
    oracle per slice.  outs maps a dtype to its device output (S * m
    elements).  Returns the number of values compared."""
    from concurrent.futures import ThreadPoolExecutor, wait, FIRST_COMPLETED

    def work(s0, cnt, got_states, got):
        st = O.streams(name, kind, base, cnt, first=s0)
        if got_states is not None:
            assert (got_states == st).all(), "%s start states %d..%d" % (name, s0, s0 + cnt)
        raw = O.fill_streams(name, st, m)
        for dtype, g in got.items():
            assert_bits_equal(g, expected(name, raw, dtype), "%s %s streams %d..%d" % (name, dtype, s0, s0 + cnt))
        return cnt * m * len(got)

    cores = _host_cores()
    done, pending = 0, set()
    with ThreadPoolExecutor(cores) as ex:
        for s0 in range(0, S, slice_streams):
            cnt = min(slice_streams, S - s0)
            got_states = None if d_states is None else \
                states_from_device(name, d_states[s0 * len(d_states) // S:(s0 + cnt) * len(d_states) // S])
            got = {dt: out_to_numpy(o[s0 * m:(s0 + cnt) * m], dt) for dt, o in outs.items()}
            pending.add(ex.submit(work, s0, cnt, got_states, got))
            while len(pending) >= 2 * cores:
                fin, pending = wait(pending, return_when=FIRST_COMPLETED)
                done += sum(f.result() for f in fin)
        done += sum(f.result() for f in pending)
    return done


@pytest.mark.parametrize("name", W.BULK_VARIANTS)
def test_bulk_configuration_full(ctx, xr, name):
    """2^20 streams x 2^10 outputs from SplitMix64(42) in the launch
    configuration the benchmark times (seed, stream starts, tile fill): every
    start state and every value, as the native word and as doubles (2^31
    values), against the oracle run on all host cores."""
    import torch
    c = W.CONFIG_BULK
    S, m = c["S"], c["m"]
    base = O.seed(name, c["seed"])
    d_base = ctx.empty_states(name, 1)
    ctx.seed(name, c["seed"], d_base)
    d_states = ctx.empty_states(name, S)
    ctx.make_streams(name, c["kind"], d_base, 0, S, d_states)
    outs = {}
    for dtype in (xr.native_dtype(name), "f64"):
        outs[dtype] = ctx.empty_output(S * m, dtype)
        ctx.fill(name, d_states, S, m, dtype, outs[dtype])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert compare_streams_in_full(name, c["kind"], base, S, m, d_states, outs) == 2 * S * m
    del outs


@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128+", "xoshiro128++"])
def test_bulk_configuration_through_fill_streams_full(ctx, xr, name):
    """2^20 streams x 2^10 outputs from SplitMix64(42) through xr_fill_streams
    (its state-table path, for these 8-KiB rows): every value, native word
    and f64, against the oracle on every host core."""
    import torch
    c = W.CONFIG_BULK
    S, m = c["S"], c["m"]
    base = O.seed(name, c["seed"])
    d_base = ctx.empty_states(name, 1)
    ctx.seed(name, c["seed"], d_base)
    outs = {}
    for dtype in (xr.native_dtype(name), "f64"):
        outs[dtype] = ctx.empty_output(S * m, dtype)
        ctx.fill_streams(name, c["kind"], d_base, 0, S, m, dtype, outs[dtype])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert compare_streams_in_full(name, c["kind"], base, S, m, None, outs) == 2 * S * m
    del outs


@pytest.mark.parametrize("kind", ["jump", "long"])
def test_jumpstart_configuration_fused_full(ctx, xr, kind):
    """The jump-start configuration in full through xr_fill_streams (start
    states computed in the generating threads, the launch the benchmark
    times): all 2^24 xoshiro256++ streams J^i(s0) / L^i(s0) x 64 u64 outputs,
    2^30 values, against one CPU jump after another on every host core."""
    import torch
    c = W.CONFIG_JUMPSTART
    name, S, m = c["variant"], c["S"], c["m"]
    base = O.seed(name, c["seed"])
    d_base = ctx.empty_states(name, 1)
    ctx.seed(name, c["seed"], d_base)
    out = ctx.empty_output(S * m, "u64")
    ctx.fill_streams(name, kind, d_base, 0, S, m, "u64", out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert compare_streams_in_full(name, kind, base, S, m, None, {"u64": out}, slice_streams=1 << 14) == S * m


@pytest.mark.parametrize("kind", ["jump", "long"])
def test_jumpstart_configuration_two_calls_full(ctx, xr, kind):
    """The same configuration through xr_make_streams and xr_fill: all 2^24
    start states of the table and all 2^30 values in full."""
    import torch
    c = W.CONFIG_JUMPSTART
    name, S, m = c["variant"], c["S"], c["m"]
    base = O.seed(name, c["seed"])
    d_base = ctx.empty_states(name, 1)
    ctx.seed(name, c["seed"], d_base)
    d_states = ctx.empty_states(name, S)
    ctx.make_streams(name, kind, d_base, 0, S, d_states)
    out = ctx.empty_output(S * m, "u64")
    ctx.fill(name, d_states, S, m, "u64", out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert compare_streams_in_full(name, kind, base, S, m, d_states, {"u64": out}, slice_streams=1 << 14) == S * m


# (S, first, m).  Below 512 x 32 streams everything goes through a state
# table; from there on chunks of 512 P streams (P a power of two) take the
# fused kernels.  Cases: tiny; below one chunk; a row length the tile store
# cannot take; one chunk (P = 32); a chunk + a tail; two chunks (P = 64, 32)
# + a tail with a high first; one chunk of P = 512 + a tail; long rows (the
# kernel that reuses its table memory as tiles) with a tail, and P = 64.
FILL_STREAMS_CASES = [(1, 0, 16), (513, 7, 64), (1024, 5, 5), (16384, 0, 64), (16384 + 5, 7, 64),
                      (3 * 16384 + 100, 2**40 + 1, 24), (2 * 256 * 512 + 3, 11, 4), (16384 + 3, 9, 1000),
                      (2 * 16384, 0, 520)]


@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoroshiro128++", "xoshiro128**",
                                  "xoroshiro64*", "xoshiro512++"])
@pytest.mark.parametrize("kind", ["jump", "long"])
def test_fill_streams(ctx, xr, name, kind):
    """xr_fill_streams (stream starts fused with the fill) against the
    oracle's J^(first + i)(base) streams and their outputs, every dtype, with
    canaries around the output."""
    import torch
    base = O.seed(name, 7)
    d_base = states_to_device(name, base[None, :])
    for S, first, m in FILL_STREAMS_CASES:
        raw = O.bulk_fill(name, kind, base, S, m, first=first).reshape(-1)
        for dtype in (xr.native_dtype(name), "f64", "f32"):
            buf, view, start, nb = guarded_output(xr, S * m, dtype)
            ctx.fill_streams(name, kind, d_base, first, S, m, dtype, as_dtype(view, dtype))
            torch.cuda.synchronize()
            check_canaries(buf, start, nb)
            got = out_to_numpy(as_dtype(view, dtype), dtype)
            assert_bits_equal(got, expected(name, raw, dtype),
                              "%s %s %s S=%d first=%d m=%d" % (name, kind, dtype, S, first, m))
    assert ctx.status() == 0


def test_fill_host_chunks(ctx, xr):
    """End-to-end call into host memory, large enough for three staging chunks."""
    import torch
    name = "xoshiro256**"
    S, m = (1 << 16) + 100, 1 << 10
    base = O.seed(name, 5)
    h_out = torch.empty(S * m, dtype=torch.int64).pin_memory()
    ctx.fill_host(name, "jump", states_to_bytes(name, base), 7, S, m, "u64", h_out)
    got = h_out.numpy().view(np.uint64).reshape(S, m)
    d = O.jump_log2(name, "jump")
    for i in W.sample_indices(S, 24, seed=5):
        raw, _ = O.generate(name, O.jump_pow(name, d, 7 + int(i), base), m)
        assert_bits_equal(got[i], raw, "stream %d" % i)


@pytest.mark.parametrize("name", ["xoshiro512++", "xoroshiro1024**", "xoroshiro64*"])
def test_fill_host_every_state_size(ctx, xr, name):
    """The host-buffer call copies the base state into the context before the
    stream starts: 64- and 128-byte states must arrive whole.  Every stream of
    a small range (a high first index) is compared with the oracle."""
    import torch
    S, m, first = 300, 40, 2**33 + 5
    base = O.seed(name, 77)
    dtype = xr.native_dtype(name)
    h_out = torch.empty(S * m, dtype=xr.torch_dtype(dtype)).pin_memory()
    ctx.fill_host(name, "long", states_to_bytes(name, base), first, S, m, dtype, h_out)
    raw = O.bulk_fill(name, "long", base, S, m, first=first).reshape(-1)
    assert_bits_equal(out_to_numpy(h_out, dtype), expected(name, raw, dtype), name)
    assert ctx.status() == 0


# ------------------------------------------------------------------ errors

def test_zero_state_is_reported(ctx, xr):
    import torch
    name = "xoroshiro128+"
    t = ctx.empty_states(name, 4)
    with pytest.raises(xr.XRError) as e:
        ctx.set_state(name, bytes(16), t)
    assert e.value.status == xr.XR_EZERO_STATE
    assert ctx.status(reset=True) == 0
    out = ctx.empty_output(4 * 8, "u64")
    ctx.fill(name, t, 4, 8, "u64", out)                # all four states are zero
    torch.cuda.synchronize()
    assert ctx.status() == xr.XR_EZERO_STATE
    assert ctx.status(reset=True) == xr.XR_EZERO_STATE
    assert ctx.status() == 0


def test_invalid_arguments(ctx, xr):
    t = ctx.empty_states("xoshiro256**", 1)
    out = ctx.empty_output(16, "u64")
    with pytest.raises(xr.XRError) as e:
        ctx.fill("xoshiro256**", t, 1, 16, "u32", out)
    assert e.value.status == xr.XR_EINVAL
    with pytest.raises(ValueError):
        ctx.fill("xoshiro256**", t, 1, 17, "u64", out)   # buffer too small


def test_fill_streams_invalid_arguments(ctx, xr):
    """xr_fill_streams rejects a dtype the generator does not have, an output
    not aligned to its element size, a misaligned base state and an unknown
    jump kind, and writes nothing; S = 0 and m = 0 are no-ops."""
    import ctypes
    import torch
    lib, h = xr.lib(), ctx.handle
    v = xr.VARIANTS["xoshiro256**"]
    base = ctx.empty_states("xoshiro256**", 2)
    ctx.seed("xoshiro256**", 1, base)
    out = torch.full((1024 + 16,), 7, dtype=torch.uint8, device="cuda")
    p, b = out.data_ptr(), base.data_ptr()
    u64, u32 = xr.DTYPES["u64"], xr.DTYPES["u32"]
    call = lambda kind, dt, base_ptr, out_ptr, S, m: lib.xr_fill_streams(h, v, kind, ctypes.c_void_p(base_ptr), 0, S, m,
                                                                         dt, ctypes.c_void_p(out_ptr), None)
    assert call(xr.KINDS["jump"], u32, b, p, 4, 16) == xr.XR_EINVAL       # no u32 outputs for a 64-bit generator
    assert call(xr.KINDS["jump"], u64, b, p + 4, 4, 16) == xr.XR_EINVAL   # output not 8-byte aligned
    assert call(xr.KINDS["jump"], u64, b + 8, p, 4, 16) == xr.XR_EINVAL   # state not 16-byte aligned
    assert call(7, u64, b, p, 4, 16) == xr.XR_EINVAL                      # no such jump kind
    assert call(xr.KINDS["jump"], u64, b, p, 0, 16) == xr.XR_OK
    assert call(xr.KINDS["jump"], u64, b, p, 4, 0) == xr.XR_OK
    # stream indices first .. first + S - 1 must fit in 64 bits (the last one may be 2^64 - 1)
    last = lambda first, S: lib.xr_fill_streams(h, v, xr.KINDS["jump"], ctypes.c_void_p(b), first, S, 16, u64,
                                                ctypes.c_void_p(p), None)
    assert last(2**64 - 3, 4) == xr.XR_EINVAL
    assert last(2**64 - 4, 4) == xr.XR_OK
    torch.cuda.synchronize()
    assert (out[512:] == 7).all()   # the last call wrote its 4 x 16 u64 and nothing past them
    want = O.bulk_fill("xoshiro256**", "jump", O.seed("xoshiro256**", 1), 4, 16, first=2**64 - 4).reshape(-1)
    assert_bits_equal(out[:512].cpu().numpy().view(np.uint64), want, "streams 2^64 - 4 .. 2^64 - 1")
    host = np.zeros(4 * 16, dtype=np.uint64)
    hb = np.frombuffer(base.cpu().numpy().tobytes()[:32], dtype=np.uint8).copy()
    assert lib.xr_fill_host(h, v, xr.KINDS["jump"], hb.ctypes.data_as(ctypes.c_void_p), 2**64 - 3, 4, 16, u64,
                            host.ctypes.data_as(ctypes.c_void_p), None) == xr.XR_EINVAL
    assert ctx.status() == 0


# ------------------------------------------------------------------ small outputs inside rows

def _state_before(name, target, k):
    """T^(-k) target: the state k steps before `target` (the period is 2^n - 1, Sec. 6)."""
    n = O.state_bits(name)
    return O.jump_pow(name, 0, (1 << n) - 1 - k, np.array(target, dtype=np.uint64))


def _small_output_starts(name, ks, xs):
    """Start states whose output k (for each k in ks) is the crafted value x."""
    starts, where = [], []
    for k in ks:
        for x in xs:
            target = [x, 0] if O.state_words(name) == 2 else [x, 0x1234567, 0x89ABCDE, 0]
            s0 = _state_before(name, target, k)
            assert int(O.generate(name, s0, k + 1)[0][k]) == x
            starts.append(s0)
            where.append((k, x))
    return np.array(starts, dtype=np.uint64), where


@pytest.mark.parametrize("name", ["xoshiro256+", "xoroshiro128+"])
def test_f64_rows_with_outputs_below_2_32(ctx, xr, name):
    """Doubles are exact when an output below 2^32 (x >> 11 has no bit in the
    high word) falls anywhere in a 16-value row, not only at a stream's first
    output: such rows are regenerated with the exact conversion."""
    import torch
    ks = [0, 15, 16, 37, 1000, 1023]
    starts, _ = _small_output_starts(name, ks, [0, 5, 2**11, 2**31 + 7, 2**32 - 1])
    S, m = len(starts), 1024
    raw = O.fill_streams(name, starts, m)
    for layout in ("stream", "interleaved"):
        out = ctx.empty_output(S * m, "f64")
        ctx.fill(name, states_to_device(name, starts), S, m, "f64", out, layout=layout)
        torch.cuda.synchronize()
        got = out_to_numpy(out, "f64")
        want = expected(name, raw, "f64")
        if layout == "interleaved":
            want = want.reshape(S, m).T.reshape(-1)
        assert_bits_equal(got, want, "f64 " + layout)


def test_batch_f64_rows_with_outputs_below_2_32(ctx, xr):
    """The same inside full batch segments (the tile path of xr_batch_run):
    requests whose slot state puts a small output at output 5000 or 20000."""
    import torch
    name = "xoshiro256+"
    starts, _ = _small_output_starts(name, [5000, 20000, 32767], [3, 2**32 - 1])
    n = 32 * 1024
    specs = [(name, "f64", n, r) for r in range(len(starts))]
    reqs, offs, arena = xr.pack_requests(specs)
    b = xr.Batch(ctx, reqs)
    slots = torch.zeros(len(specs) * 32, dtype=torch.uint8)
    for r, s0 in enumerate(starts):
        slots[r * 32:(r + 1) * 32] = torch.from_numpy(s0.astype(np.uint64).view(np.uint8).copy())
    d_slots = slots.cuda()
    out = torch.zeros(arena, dtype=torch.uint8, device="cuda")
    b.run(None, d_slots, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for r, s0 in enumerate(starts):
        raw, _ = O.generate(name, s0, n)
        assert_bits_equal(o[offs[r]:offs[r] + n * 8].view(np.float64), expected(name, raw, "f64"), "request %d" % r)
    b.close()
