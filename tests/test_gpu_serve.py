"""Serving with continuous batching (xr_server_*): device-resident client
states continue across requests, results in the mix equal each client's
sequence alone, admission respects the output budget.  Bit-exact throughout."""
import threading

import numpy as np
import pytest

import oracle as O
import workloads as W
from xr_testutil import assert_bits_equal, expected

pytestmark = pytest.mark.gpu

NP = {"u64": np.uint64, "u32": np.uint32, "f64": np.float64, "f32": np.float32}


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


CLIENTS = ["xoshiro256**", "xoroshiro128++", "xoshiro256+", "xoroshiro128**", "xoshiro128++", "xoshiro128**",
           "xoshiro256++", "xoroshiro128+", "xoroshiro128*", "xoroshiro64**"]


def mixed_trace(nreq, seed, max_len=1 << 17, clients=CLIENTS):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nreq):
        c = int(rng.integers(0, len(clients)))
        name = clients[c]
        dt = [W.native_dtype(name), "f64", "f32"][int(rng.integers(0, 3))]
        n = int(np.floor(np.exp(rng.uniform(0, np.log(max_len)))))
        out.append((c, max(n, 1), dt))
    return out


class Expect:
    """Each client's sequence from its SplitMix64 seed, consumed in order."""

    def __init__(self, seeds, clients=CLIENTS):
        self.clients = clients
        self.state = {c: O.seed(name, seeds[c]) for c, name in enumerate(clients)}

    def take(self, c, n, dt):
        raw, self.state[c] = O.generate(self.clients[c], self.state[c], n)
        return expected(self.clients[c], raw, dt)


def read(srv, off, n, dt, torch):
    es = 8 if dt in ("u64", "f64") else 4
    buf = torch.empty(n * es, dtype=torch.uint8)
    srv.read(off, n * es, buf)
    return buf.numpy().view(NP[dt])


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_results_equal_each_client_sequence(ctx, xr, mode):
    """Requests submitted in bursts while earlier ones run: every output is the
    client's next values, exactly as if its requests ran alone in order."""
    import torch
    seeds = [101 + c for c in range(len(CLIENTS))]
    trace = mixed_trace(240, seed=31)
    exp = Expect(seeds)
    with xr.Server(ctx, CLIENTS, seeds, arena_bytes=1 << 30, mode=mode, max_rounds=3,
                   max_round_requests=64) as srv:
        for burst in range(0, len(trace), 40):
            tickets = [(srv.submit(c, n, dt), c, n, dt) for (c, n, dt) in trace[burst:burst + 40]]
            for t, c, n, dt in tickets:
                off, lat = srv.wait(t)
                assert lat >= 0
                assert_bits_equal(read(srv, off, n, dt, torch), exp.take(c, n, dt), "client %d n=%d" % (c, n))
                srv.release(t)
        for c, name in enumerate(CLIENTS):
            want = exp.state[c].astype(np.uint32 if O.word_bits(name) == 32 else np.uint64).tobytes()
            assert srv.client_state(c) == want
        st = srv.stats()
        assert st["completed"] == len(trace) and st["released"] == len(trace)
        if mode == "batched":
            assert st["rounds"] >= 2
    assert ctx.status() == 0


def test_admission_waits_for_memory(ctx, xr):
    """A 4 MiB budget and 120 requests of up to 1 MiB each submitted at once:
    admission holds requests until released space allows them; all complete
    and the arena never exceeds the budget."""
    import torch
    seeds = list(range(len(CLIENTS)))
    rng = np.random.default_rng(7)
    n = rng.integers(1000, 1 << 17, size=120).astype(np.uint64)
    clients = rng.integers(0, len(CLIENTS), size=120).astype(np.uint32)
    dts = ["f64"] * 120
    with xr.Server(ctx, CLIENTS, seeds, arena_bytes=4 << 20, mode="batched", max_rounds=2) as srv:
        lat, wall = srv.replay(np.zeros(120), clients, n, dts)
        st = srv.stats()
        assert st["completed"] == 120 and st["arena_peak"] <= 4 << 20
        assert (lat > 0).all() and wall > 0
        # the states moved on by exactly the requested counts
        exp = Expect(seeds)
        for c, k in zip(clients, n):
            exp.take(int(c), int(k), "f64")
        for c, name in enumerate(CLIENTS):
            want = exp.state[c].astype(np.uint32 if O.word_bits(name) == 32 else np.uint64).tobytes()
            assert srv.client_state(c) == want


def test_concurrent_submitters(ctx, xr):
    """Two host threads submit for disjoint clients at the same time."""
    import torch
    seeds = [9 + c for c in range(len(CLIENTS))]
    out = {}

    def worker(cl, srv, tid):
        got = []
        for k in range(30):
            c = cl[k % len(cl)]
            n = 500 + 37 * k
            t = srv.submit(c, n, "f64")
            got.append((t, c, n))
        res = []
        for t, c, n in got:
            off, _ = srv.wait(t)
            res.append((c, n, read(srv, off, n, "f64", torch).copy()))
            srv.release(t)
        out[tid] = res

    with xr.Server(ctx, CLIENTS, seeds, arena_bytes=64 << 20, mode="batched", max_rounds=3) as srv:
        th = [threading.Thread(target=worker, args=([0, 2, 4, 6], srv, 0)),
              threading.Thread(target=worker, args=([1, 3, 5, 7], srv, 1))]
        for t in th:
            t.start()
        for t in th:
            t.join()
    exp = Expect(seeds)
    for tid in (0, 1):
        for c, n, got in out[tid]:
            assert_bits_equal(got, exp.take(c, n, "f64"), "client %d" % c)


def test_rejects_bad_requests(ctx, xr):
    with xr.Server(ctx, CLIENTS, list(range(len(CLIENTS))), arena_bytes=1 << 20) as srv:
        with pytest.raises(xr.XRError):
            srv.submit(len(CLIENTS), 10, "f64")          # no such client
        with pytest.raises(xr.XRError):
            srv.submit(4, 10, "u64")                     # 32-bit client, u64 output
        with pytest.raises(xr.XRError):
            srv.submit(0, 1 << 20, "u64")                # larger than the arena
        with pytest.raises(xr.XRError):
            srv.release(12345)


LARGE_CLIENTS = ["xoroshiro1024++", "xoshiro512**", "xoshiro256**", "xoroshiro1024*", "xoshiro512+",
                 "xoroshiro64*", "xoshiro128++", "xoroshiro1024**"]


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_large_state_clients(ctx, xr, mode):
    """Clients of xoshiro512 and xoroshiro1024 (64- and 128-byte states, Sec.
    3.1 X_kw and Sec. 3.2 S_8w) served beside smaller ones: every output is
    the client's next values, and each client's resident state has moved on
    by exactly its requests."""
    import torch
    seeds = [40 + c for c in range(len(LARGE_CLIENTS))]
    trace = mixed_trace(120, seed=33, max_len=1 << 16, clients=LARGE_CLIENTS)
    trace += [(0, 70000, "f64"), (1, 3 * 1024, "u64"), (3, 1, "f32")]
    exp = Expect(seeds, LARGE_CLIENTS)
    with xr.Server(ctx, LARGE_CLIENTS, seeds, arena_bytes=256 << 20, mode=mode, max_rounds=3,
                   max_round_requests=32) as srv:
        for burst in range(0, len(trace), 30):
            tickets = [(srv.submit(c, n, dt), c, n, dt) for (c, n, dt) in trace[burst:burst + 30]]
            for t, c, n, dt in tickets:
                off, _ = srv.wait(t)
                assert_bits_equal(read(srv, off, n, dt, torch), exp.take(c, n, dt),
                                  "%s client %d n=%d" % (LARGE_CLIENTS[c], c, n))
                srv.release(t)
        for c, name in enumerate(LARGE_CLIENTS):
            want = exp.state[c].astype(np.uint32 if O.word_bits(name) == 32 else np.uint64).tobytes()
            assert srv.client_state(c) == want, name
    assert ctx.status() == 0


def test_serving_trace_sampled(ctx, xr):
    """A short serving trace (256 clients, Poisson arrivals, 2^10 .. 2^20
    values) through replay; then the final client states against the oracle."""
    names, seeds = W.serve_clients(256)
    arr, cl, n, dt = W.serve_trace(400, nclients=256, rate=20000.0, max_len=1 << 20, trace_seed=8)
    with xr.Server(ctx, names, seeds, arena_bytes=1 << 30, mode="batched") as srv:
        lat, wall = srv.replay(arr, cl, n, dt)
        assert len(lat) == 400 and (lat > 0).all()
        total = {}
        for c, k in zip(cl, n):
            total[int(c)] = total.get(int(c), 0) + int(k)
        for c in list(total)[:40]:
            st = O.jump_pow(names[c], 0, total[c], O.seed(names[c], seeds[c]))
            want = st.astype(np.uint64).tobytes()
            assert srv.client_state(c) == want, c


def test_bounded_wait(ctx, xr):
    """xr_server_wait_for: a request still running returns XR_ETIMEOUT (None
    here) and stays valid; waiting again completes it with the right outputs."""
    import torch
    seeds = [3 + c for c in range(len(CLIENTS))]
    with xr.Server(ctx, CLIENTS, seeds, arena_bytes=1 << 31, mode="batched") as srv:
        big = srv.submit(0, 1 << 27, "f64")      # 1 GiB: still running right after submission
        assert srv.wait(big, timeout_us=0) is None
        off, lat = srv.wait(big, timeout_us=60e6)
        got = read(srv, off, 1 << 27, "f64", torch)
        assert_bits_equal(got[:4096], Expect(seeds).take(0, 4096, "f64"), "head")
        assert srv.wait(big, timeout_us=0) is not None      # complete: no timeout
        srv.release(big)
        with pytest.raises(xr.XRError):
            srv.wait(big + 1000, timeout_us=1.0)            # no such ticket
        with pytest.raises(xr.XRError):
            srv.wait(big, timeout_us=-1.0)                  # bad limit
