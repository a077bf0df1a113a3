"""Stream starts under CUDA stream capture (include/xr.h, xr_make_streams and
xr_fill_streams): a call being captured never builds a power set or grows
the scratch (that would allocate and wait for the device); it takes the path
that needs neither, with the same results.  Bit-exact against the oracle."""
import numpy as np
import pytest

import oracle as O
from xr_testutil import assert_bits_equal, states_from_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xr():
    from paper_1805_01407_gb300 import build
    build.build()
    import paper_1805_01407_gb300 as xr
    return xr


def _capture(torch, fn):
    """fn() captured into a CUDA graph on a side stream; returns the graph."""
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    return g


@pytest.mark.parametrize("kind", ["jump", "long"])
def test_fill_streams_captured_before_and_after_its_power_set(xr, kind):
    import torch
    name, S, m = "xoshiro256++", 16384 + 5, 24     # one chunk of 512 x 32 streams and a tail
    base = O.seed(name, 21)
    want = O.bulk_fill(name, kind, base, S, m).reshape(-1)
    with xr.Context(0) as ctx:                      # fresh: no power set of the chunk distance yet
        d_base = ctx.empty_states(name, 1)
        ctx.seed(name, 21, d_base)
        # grow the shared scratch outside capture with a generator that builds no power set
        big = "xoshiro512+"
        b2 = ctx.empty_states(big, 1)
        ctx.seed(big, 3, b2)
        tmp = ctx.empty_output(16383 * 8, "u64")
        ctx.fill_streams(big, kind, b2, 0, 16383, 8, "u64", tmp)
        torch.cuda.synchronize()
        out = torch.zeros(S * m, dtype=torch.int64, device="cuda")
        # an allocation or a device-wide wait inside the call would invalidate the capture
        g = _capture(torch, lambda: ctx.fill_streams(name, kind, d_base, 0, S, m, "u64", out))
        g.replay()
        torch.cuda.synchronize()
        assert_bits_equal(out.cpu().numpy().view(np.uint64), want, "captured, state-table path")
        # outside capture the call builds the power set and fuses; captured again, it reuses it
        out.zero_()
        ctx.fill_streams(name, kind, d_base, 0, S, m, "u64", out)
        torch.cuda.synchronize()
        assert_bits_equal(out.cpu().numpy().view(np.uint64), want, "fused path")
        out.zero_()
        g2 = _capture(torch, lambda: ctx.fill_streams(name, kind, d_base, 0, S, m, "u64", out))
        g2.replay()
        g2.replay()
        torch.cuda.synchronize()
        assert_bits_equal(out.cpu().numpy().view(np.uint64), want, "captured, fused path")
        assert ctx.status() == 0


def test_make_streams_captured_without_its_power_set(xr):
    import torch
    name, S = "xoroshiro128**", 16384 * 2 + 9
    base = O.seed(name, 8)
    want = O.streams(name, "jump", base, S, first=5)
    with xr.Context(0) as ctx:
        d_base = ctx.empty_states(name, 1)
        ctx.seed(name, 8, d_base)
        states = ctx.empty_states(name, S)
        g = _capture(torch, lambda: ctx.make_streams(name, "jump", d_base, 5, S, states))
        g.replay()
        torch.cuda.synchronize()
        assert (states_from_device(name, states) == want).all()
        states.zero_()
        ctx.make_streams(name, "jump", d_base, 5, S, states)   # builds the power set, chunked path
        torch.cuda.synchronize()
        assert (states_from_device(name, states) == want).all()
        assert ctx.status() == 0
