"""Batched uneven requests in one persistent launch (xr_batch_*), against the
oracle and against each request run alone through xr_fill_seq.

Every comparison is bit-exact (integer outputs and exact conversions)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from xr_testutil import assert_bits_equal, expected

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


def slot_state(name, slots_np, slot, slot_bytes=32):
    """Oracle words of a state slot (uint8 numpy array of all slots)."""
    k, w = O.state_words(name), O.word_bits(name)
    b = slots_np[slot * slot_bytes: slot * slot_bytes + k * w // 8].tobytes()
    return np.frombuffer(b, dtype=np.uint32 if w == 32 else np.uint64).astype(np.uint64)


def request_view(out_np, off, n, dtype):
    es = 8 if dtype in ("u64", "f64") else 4
    npd = {"u64": np.uint64, "u32": np.uint32, "f64": np.float64, "f32": np.float32}[dtype]
    return out_np[off: off + n * es].view(npd)


def small_mix(nreq, max_len, seed, variants=W.SLOT_VARIANTS):
    rng = np.random.default_rng(seed)
    specs = []
    for r in range(nreq):
        name = variants[int(rng.integers(0, len(variants)))]
        dt = [W.native_dtype(name), "f64", "f32"][int(rng.integers(0, 3))]
        n = int(np.clip(np.floor(np.exp(rng.uniform(0, np.log(max_len + 1)))), 0, max_len))
        if r % 17 == 0:
            n = 0
        specs.append((name, dt, n, r))
    return specs


def run_batch(xr, ctx, specs, seeds, use_graph=False, tune=False, reps=1):
    import torch
    reqs, offs, arena = xr.pack_requests(specs)
    b = xr.Batch(ctx, reqs)
    assert b.arena_bytes <= arena
    slots = torch.zeros(len(specs) * b.slot_bytes, dtype=torch.uint8, device="cuda")
    out = torch.full((max(arena, 16),), 0x5A, dtype=torch.uint8, device="cuda")
    d_seeds = torch.tensor(seeds, dtype=torch.int64, device="cuda") if seeds is not None else None
    if tune:
        # the tuner restores the slots it started from
        if d_seeds is not None:
            b.run(d_seeds, slots, out)
        before = slots.clone()
        b.tune(None, slots, out)
        assert torch.equal(before, slots)
        d_seeds = None
        reps = 1
    for k in range(reps):
        b.run(d_seeds if k == 0 else None, slots, out, use_graph=use_graph)
    torch.cuda.synchronize()
    return b, offs, out.cpu().numpy(), slots.cpu().numpy()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(ctx, xr, use_graph):
    specs = small_mix(300, 1 << 14, seed=21)
    seeds = [1000 + r for r in range(len(specs))]
    b, offs, out, slots = run_batch(xr, ctx, specs, seeds, use_graph=use_graph)
    for r, (name, dt, n, slot) in enumerate(specs):
        s0 = O.seed(name, seeds[r])
        raw, after = O.generate(name, s0, n)
        assert_bits_equal(request_view(out, offs[r], n, dt), expected(name, raw, dt), "request %d" % r)
        assert (slot_state(name, slots, slot) == after).all(), r
    assert ctx.status() == 0
    b.close()


def test_batch_continues_sequences_across_runs(ctx, xr):
    """A seeded run, then two runs of one captured graph (the second is a
    replay): every slot's sequence continues, so the last run gives outputs
    2n .. 3n-1."""
    import torch
    specs = small_mix(120, 5000, seed=22)
    seeds = list(range(len(specs)))
    reqs, offs, arena = xr.pack_requests(specs)
    b = xr.Batch(ctx, reqs)
    slots = torch.zeros(len(specs) * 32, dtype=torch.uint8, device="cuda")
    out = torch.zeros(max(arena, 16), dtype=torch.uint8, device="cuda")
    b.run(torch.tensor(seeds, dtype=torch.int64, device="cuda"), slots, out)
    b.run(None, slots, out, use_graph=True)
    b.run(None, slots, out, use_graph=True)
    torch.cuda.synchronize()
    o, sl = out.cpu().numpy(), slots.cpu().numpy()
    for r, (name, dt, n, slot) in enumerate(specs):
        raw, after = O.generate(name, O.seed(name, seeds[r]), 3 * n)
        assert_bits_equal(request_view(o, offs[r], n, dt), expected(name, raw[2 * n:], dt), "request %d" % r)
        assert (slot_state(name, sl, slot) == after).all()
    b.close()


def test_batch_alone_equals_in_the_mix(ctx, xr):
    """Each request of a mixed batch equals the same request run alone through
    xr_fill_seq (seeded the same way)."""
    import torch
    specs = small_mix(200, 1 << 16, seed=23)
    seeds = [7 * r + 3 for r in range(len(specs))]
    b, offs, out, slots = run_batch(xr, ctx, specs, seeds, use_graph=True)
    for r, (name, dt, n, slot) in enumerate(specs):
        st = ctx.empty_states(name, 1)
        ctx.seed(name, seeds[r], st)
        alone = ctx.empty_output(max(n, 1), dt)
        ctx.fill_seq(name, st, n, dt, alone)
        torch.cuda.synchronize()
        got = request_view(out, offs[r], n, dt)
        assert_bits_equal(got, alone.cpu().numpy().view(got.dtype)[:n], "request %d" % r)
    b.close()


def test_batch_tuner_keeps_results(ctx, xr):
    specs = small_mix(150, 1 << 13, seed=24)
    seeds = list(range(500, 500 + len(specs)))
    b, offs, out, slots = run_batch(xr, ctx, specs, seeds, tune=True)
    opt, block = b.get_config()
    assert opt in (4, 8, 16, 32, 64) and block in (128, 256, 512)
    # after tuning the batch ran once more from the seeded slots: outputs n .. 2n-1
    for r, (name, dt, n, slot) in enumerate(specs):
        raw, after = O.generate(name, O.seed(name, seeds[r]), 2 * n)
        assert_bits_equal(request_view(out, offs[r], n, dt), expected(name, raw[n:], dt), "request %d" % r)
    b.close()


@pytest.mark.parametrize("opt,block,align", [(4, 128, None), (8, 512, None), (16, 256, 256), (32, 256, None),
                                             (64, 128, 16)])
def test_batch_every_config(ctx, xr, opt, block, align):
    """Every tuner configuration, with requests placed on row boundaries (tile
    stores for full segments) or only on 16/256-byte boundaries (per-lane
    bulk copies everywhere)."""
    import torch
    specs = small_mix(60, 3000, seed=25) + [("xoshiro256**", "u64", 40000, 60), ("xoshiro128++", "f32", 70000, 61),
                                            ("xoroshiro128+", "f64", 33 * 1024, 62),
                                            ("xoshiro512+", "f64", 34 * 1024 + 3, 63),
                                            ("xoroshiro1024++", "u64", 2049, 64)]
    reqs, offs, arena = xr.pack_requests(specs, align=align)
    b = xr.Batch(ctx, reqs)
    b.set_config(opt, block)
    slots = torch.zeros(len(specs) * b.slot_bytes, dtype=torch.uint8, device="cuda")
    out = torch.zeros(max(arena, 16), dtype=torch.uint8, device="cuda")
    seeds = torch.arange(len(specs), dtype=torch.int64, device="cuda") + 77
    b.run(seeds, slots, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for r, (name, dt, n, slot) in enumerate(specs):
        raw, _ = O.generate(name, O.seed(name, 77 + r), n)
        assert_bits_equal(request_view(o, offs[r], n, dt), expected(name, raw, dt), "request %d" % r)
    b.close()


def test_batch_rejects_bad_plans(ctx, xr):
    R = xr.Request
    with pytest.raises(xr.XRError):
        xr.Batch(ctx, [R(0, 0, 10, 0, 0), R(1, 0, 10, 0, 256)])          # slot used twice
    with pytest.raises(xr.XRError):
        xr.Batch(ctx, [R(0, 0, 10, 0, 8)])                                # unaligned offset
    with pytest.raises(xr.XRError):
        xr.Batch(ctx, [R(6, 0, 10, 0, 0)])                                # u64 from a 32-bit generator


def test_batch_slot_bytes_follow_the_largest_state(ctx, xr):
    """Slots are 32 bytes unless a request's state is larger: 64 with a
    xoshiro512 request, 128 with a xoroshiro1024 request."""
    R, V = xr.Request, xr.VARIANTS
    for names, want in ((["xoshiro256**", "xoroshiro64*"], 32), (["xoshiro128+", "xoshiro512**"], 64),
                        (["xoshiro512+", "xoroshiro1024++", "xoroshiro128+"], 128)):
        b = xr.Batch(ctx, [R(V[nm], 2, 10, k, 256 * k) for k, nm in enumerate(names)])
        assert b.slot_bytes == want, names
        b.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_large_states_alone_and_in_the_mix(ctx, xr, use_graph):
    """Requests of all 18 generators, xoshiro512 and xoroshiro1024 among them
    (Sec. 3.1 X_kw, Fig. 2; Sec. 3.2 S_8w, Fig. 4), in one batch with
    128-byte slots: each equals the oracle and the same request alone through
    xr_fill_seq; the slots hold the advanced states; a second run (a graph
    replay when use_graph) continues every sequence."""
    import torch
    specs = small_mix(160, 70000, seed=26, variants=W.ALL_VARIANTS)
    specs += [("xoshiro512++", "f64", 40 * 1024, 160), ("xoroshiro1024**", "u64", 33 * 1024 + 5, 161),
              ("xoroshiro1024*", "f32", 1, 162), ("xoshiro512**", "u64", 300000, 163)]
    seeds = [3 * r + 11 for r in range(len(specs))]
    b, offs, out, slots = run_batch(xr, ctx, specs, seeds, use_graph=use_graph)
    assert b.slot_bytes == 128
    for r, (name, dt, n, slot) in enumerate(specs):
        raw, after = O.generate(name, O.seed(name, seeds[r]), n)
        assert_bits_equal(request_view(out, offs[r], n, dt), expected(name, raw, dt), "request %d %s" % (r, name))
        assert (slot_state(name, slots, slot, 128) == after).all(), (r, name)
        st = ctx.empty_states(name, 1)
        ctx.seed(name, seeds[r], st)
        alone = ctx.empty_output(max(n, 1), dt)
        ctx.fill_seq(name, st, n, dt, alone)
        torch.cuda.synchronize()
        got = request_view(out, offs[r], n, dt)
        assert_bits_equal(got, alone.cpu().numpy().view(got.dtype)[:n], "request %d alone" % r)
    # second run from the advanced slots
    d_slots = torch.from_numpy(slots.copy()).cuda()
    d_out = torch.zeros(len(out), dtype=torch.uint8, device="cuda")
    b.run(None, d_slots, d_out, use_graph=use_graph)
    torch.cuda.synchronize()
    o2 = d_out.cpu().numpy()
    for r, (name, dt, n, slot) in enumerate(specs):
        if n > 5000 and r % 7:
            continue   # the oracle's 2n outputs of the long ones: a sample suffices
        raw, _ = O.generate(name, O.seed(name, seeds[r]), 2 * n)
        assert_bits_equal(request_view(o2, offs[r], n, dt), expected(name, raw[n:], dt), "request %d run 2" % r)
    assert ctx.status() == 0
    b.close()


def oracle_requests_in_full(specs, seeds, out_np, offs, chunk=1 << 20):
    """Every output of every request against the oracle: requests are cut into
    chunks of `chunk` values whose start states the oracle reaches by its jump
    polynomial (x^(k chunk) mod p), and the chunks run on every host core
    (worker threads; the oracle's C calls release the GIL).  Returns the
    number of values compared."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    def work(r, k0):
        name, dt, n, _ = specs[r]
        cnt = min(chunk, n - k0)
        st = O.jump_pow(name, 0, k0, O.seed(name, seeds[r])) if k0 else O.seed(name, seeds[r])
        raw, _ = O.generate(name, st, cnt)
        es = 8 if dt in ("u64", "f64") else 4
        got = request_view(out_np, offs[r] + k0 * es, cnt, dt)
        assert_bits_equal(got, expected(name, raw, dt), "request %d values %d..%d" % (r, k0, k0 + cnt))
        return cnt

    tasks = [(r, k0) for r, (_, _, n, _) in enumerate(specs) for k0 in range(0, n, chunk)]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with ThreadPoolExecutor(cores) as ex:
        return sum(ex.map(lambda t: work(*t), tasks))


def test_batch_configuration_full(ctx, xr):
    """The batched configuration (4096 requests, lengths log-uniform up to 2^24,
    8 generators, native/double, SplitMix64(r) seeds; 30 GB) in one graph
    launch: every request equals the same request run alone through
    xr_fill_seq, and every value of every request equals the oracle."""
    import torch
    specs = W.batch_requests()
    seeds = [s for (_, _, _, s) in specs]
    specs = [(v, dt, n, r) for r, (v, dt, n, _) in enumerate(specs)]
    reqs, offs, arena = xr.pack_requests(specs)
    b = xr.Batch(ctx, reqs)
    slots = torch.zeros(len(specs) * b.slot_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty(arena, dtype=torch.uint8, device="cuda")
    d_seeds = torch.tensor(seeds, dtype=torch.int64, device="cuda")
    b.run(d_seeds, slots, out, use_graph=True)
    alone = torch.empty(arena, dtype=torch.uint8, device="cuda")
    st = ctx.empty_states("xoshiro256**", 1)
    for r, (name, dt, n, _) in enumerate(specs):
        ctx.seed(name, seeds[r], st)
        ctx.fill_seq(name, st, n, dt, alone[offs[r]:].view(xr.torch_dtype(dt))[:n])
    torch.cuda.synchronize()
    for r, (name, dt, n, _) in enumerate(specs):
        a, z = offs[r], offs[r] + n * xr.dtype_bytes(dt)
        assert torch.equal(out[a:z], alone[a:z]), "request %d differs from its run alone" % r
    del alone
    o = out.cpu().numpy()
    assert oracle_requests_in_full(specs, seeds, o, offs) == sum(n for (_, _, n, _) in specs)
    assert ctx.status() == 0
    b.close()
