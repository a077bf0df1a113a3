"""The seeded input generators: sampled indices, and the recipes of the
batched and serving configurations (lengths, generators, output types,
arrival rate)."""
import numpy as np

import workloads as W


def test_sample_indices_include_both_ends():
    for S, count in ((2**24, 4096), (2**20, 66), (1000, 40), (10, 3), (5, 5), (5, 9), (3, 2)):
        idx = W.sample_indices(S, count, seed=1)
        assert len(idx) == min(count, S)
        assert (np.diff(idx) > 0).all() and idx[0] == 0 and idx[-1] == S - 1
        assert (W.sample_indices(S, count, seed=1) == idx).all()


def test_sample_indices_are_spread_over_the_range():
    idx = W.sample_indices(2**24, 4096, seed=1)
    counts = np.histogram(idx, bins=8, range=(0, 2**24))[0]
    assert counts.min() > 4096 / 8 * 0.8


def test_batch_requests_recipe():
    specs = W.batch_requests(**W.CONFIG_BATCH)
    assert len(specs) == 4096
    n = np.array([s[2] for s in specs])
    assert n.min() >= 1 and n.max() <= 1 << 24
    # log-uniform: about a quarter of the requests in each quarter of [0, 24] in log2
    q = np.histogram(np.log2(n), bins=4, range=(0, 24))[0]
    assert q.min() > 4096 / 4 * 0.8
    assert {s[0] for s in specs} == set(W.BULK_VARIANTS)
    assert {s[1] for s in specs} == {"u64", "u32", "f64"}
    assert [s[3] for s in specs] == list(range(4096))


def test_serve_trace_recipe():
    c = W.CONFIG_SERVE
    arr, cl, n, dt = W.serve_trace(20000, **c)
    rate = (len(arr) - 1) / (arr[-1] - arr[0]) * 1e6
    assert abs(rate - c["rate"]) / c["rate"] < 0.03
    assert n.min() >= c["min_len"] and n.max() <= c["max_len"]
    assert cl.max() < c["nclients"] and set(dt) == {"u64", "f64"}
    names, seeds = W.serve_clients(c["nclients"])
    assert set(names) == {"xoshiro256**", "xoroshiro128++"} and seeds == list(range(c["nclients"]))
