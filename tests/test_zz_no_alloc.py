"""GPU test of xr_fill_seq_noalloc.

That entry point serves callers that cannot allocate device memory while they
run -- code working inside an application-owned memory pool, or in a real-time
or callback path where cudaMalloc/cudaFree would block, synchronize the device
or fail.  It must give exactly what xr_fill_seq gives (outputs and advanced
state), call after call, without allocating.  This file is collected last so a
failure here cannot hide the other GPU tests; it builds its own context and
passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_OUTPUTS = 1 << 26   # XR_NOALLOC_MAX_OUTPUTS in include/xr.h
SCRATCH_BYTES = 2 << 20  # XR_NOALLOC_SCRATCH_BYTES: one state per 1024 outputs


def max_outputs_for(state_bytes):
    """XR_NOALLOC_MAX_OUTPUTS_FOR: 2^26 up to 32-byte states, then as many
    1024-output segments as the array holds states."""
    return MAX_OUTPUTS if state_bytes <= 32 else (SCRATCH_BYTES // state_bytes) << 10


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1805_01407_gb300 import build
    build.build()
    import paper_1805_01407_gb300 as xr
    f = xr.lib().xr_fill_seq_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    ctx = xr.Context(0)
    yield xr, ctx, f, torch
    ctx.close()


def _call(env, name, state, n, dtype, out):
    xr, ctx, f, torch = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(ctx.handle, xr.VARIANTS[name], state.data_ptr(), n, xr.DTYPES[dtype], out.data_ptr(),
             stream)


def _bits(t):
    a = t.cpu().numpy()
    return a.view({1: np.uint8, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128++", "xoshiro128++"])
def test_matches_fill_seq_on_two_calls_in_a_row(env, name):
    xr, ctx, f, torch = env
    for n in (1, 1000, 1024, 4097, 300001):
        for dtype in (xr.native_dtype(name), "f64"):
            a = ctx.empty_states(name, 1)
            b = ctx.empty_states(name, 1)
            ctx.seed(name, 2024, a)
            ctx.seed(name, 2024, b)
            for call in range(2):
                out_a = ctx.empty_output(n, dtype)
                out_b = ctx.empty_output(n, dtype)
                assert _call(env, name, a, n, dtype, out_a) == xr.XR_OK
                ctx.fill_seq(name, b, n, dtype, out_b)
                torch.cuda.synchronize()
                # the conversions are exact, so the tolerance is zero: equal bits
                assert (_bits(out_a) == _bits(out_b)).all(), (name, n, dtype, call)
                assert ctx.get_state(name, a) == ctx.get_state(name, b), (name, n, dtype, call)
    assert ctx.status() == 0


def test_largest_size_and_no_device_allocation(env):
    xr, ctx, f, torch = env
    name, n = "xoshiro256++", MAX_OUTPUTS
    a = ctx.empty_states(name, 1)
    b = ctx.empty_states(name, 1)
    ctx.seed(name, 7, a)
    ctx.seed(name, 7, b)
    out_a = ctx.empty_output(n, "u64")
    out_b = ctx.empty_output(n, "u64")
    assert _call(env, name, a, n, "u64", out_a) == xr.XR_OK      # first call on the device
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(env, name, a, n, "u64", out_a) == xr.XR_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for _ in range(3):
        ctx.fill_seq(name, b, n, "u64", out_b)
    torch.cuda.synchronize()
    assert (_bits(out_a) == _bits(out_b)).all()
    assert ctx.get_state(name, a) == ctx.get_state(name, b)


def test_rejects_sizes_beyond_the_maximum(env):
    xr, ctx, f, torch = env
    name = "xoroshiro128+"
    st = ctx.empty_states(name, 1)
    ctx.seed(name, 1, st)
    before = ctx.get_state(name, st)
    out = torch.full((16,), 7, dtype=torch.int64, device="cuda")
    assert _call(env, name, st, MAX_OUTPUTS + 1, "u64", out) == xr.XR_EINVAL
    torch.cuda.synchronize()
    assert (out.cpu() == 7).all() and ctx.get_state(name, st) == before


@pytest.mark.parametrize("name", ["xoshiro512++", "xoroshiro1024**"])
def test_large_states_at_their_largest_size(env, name):
    """States of 64 and 128 bytes take more of the array per segment, so their
    largest call is 2^25 and 2^24 outputs.  On a context that has not built
    the engine's jump tables yet the call refuses (building them would
    allocate) and allocates nothing; after another call has built them it
    matches xr_fill_seq at the largest size, twice in a row; one more output
    is refused with the outputs and the state untouched."""
    xr, _, f, torch = env
    sb = xr.state_bytes(name)
    n = max_outputs_for(sb)
    assert n == {64: 1 << 25, 128: 1 << 24}[sb]
    with xr.Context(0) as ctx:
        fresh = (xr, ctx, f, torch)
        a = ctx.empty_states(name, 1)
        b = ctx.empty_states(name, 1)
        ctx.seed(name, 99, a)
        ctx.seed(name, 99, b)
        out_a = ctx.empty_output(n + 1, "u64")
        out_b = ctx.empty_output(n, "u64")
        small = ctx.empty_states("xoshiro256**", 1)
        ctx.seed("xoshiro256**", 1, small)
        assert _call(fresh, "xoshiro256**", small, 16, "u64", out_b) == xr.XR_OK   # loads the array
        torch.cuda.synchronize()
        out_a.fill_(7)
        free_before = torch.cuda.mem_get_info()[0]
        before = ctx.get_state(name, a)
        assert _call(fresh, name, a, 1000, "u64", out_a) == xr.XR_EUNSUPPORTED
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert (out_a.cpu() == 7).all() and ctx.get_state(name, a) == before
        # xr_fill_seq builds the tables and grows its scratch to this size (both allocate)
        ctx.fill_seq(name, b, n, "u64", out_b)
        ctx.seed(name, 99, b)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for call in range(2):
            assert _call(fresh, name, a, n, "u64", out_a[:n]) == xr.XR_OK
            ctx.fill_seq(name, b, n, "u64", out_b)
            torch.cuda.synchronize()
            assert (_bits(out_a[:n]) == _bits(out_b)).all(), (name, call)
            assert ctx.get_state(name, a) == ctx.get_state(name, b), (name, call)
        assert torch.cuda.mem_get_info()[0] == free_before
        out_a.fill_(7)
        before = ctx.get_state(name, a)
        assert _call(fresh, name, a, n + 1, "u64", out_a) == xr.XR_EINVAL
        torch.cuda.synchronize()
        assert (out_a.cpu() == 7).all() and ctx.get_state(name, a) == before
        assert ctx.status() == 0


def test_no_allocation_in_calls_of_every_state_size(env):
    """Repeated calls of 8- to 128-byte states leave the device's free memory
    unchanged once their jump tables exist."""
    xr, ctx, f, torch = env
    names = ["xoroshiro64**", "xoroshiro128+", "xoshiro256+", "xoshiro512**", "xoroshiro1024*"]
    states, outs = {}, {}
    for name in names:
        st = ctx.empty_states(name, 1)
        ctx.seed(name, 5, st)
        ctx.jump(name, "jump", st, 1)        # builds the large engines' tables
        states[name] = st
        outs[name] = ctx.empty_output(70000, xr.native_dtype(name))
    torch.cuda.synchronize()
    assert _call(env, names[0], states[names[0]], 10, xr.native_dtype(names[0]), outs[names[0]]) == xr.XR_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for name in names:
            assert _call(env, name, states[name], 70000, xr.native_dtype(name), outs[name]) == xr.XR_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert ctx.status() == 0
