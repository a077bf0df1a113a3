"""The multi-rank path of bench.py on CPU: two gloo ranks, each owning a
disjoint range of stream indices (no collective on the data path), and the
slowest-rank timing reduction.  The shards, generated by the oracle, must
equal the single-rank result for all streams."""
import os
import socket

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    name, S, m = "xoshiro256**", 24, 16
    first = bench.shard_first(rank, S)
    base = O.seed(name, 42)
    mine = O.bulk_fill(name, "jump", base, S, m, first=first)
    slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    if rank == 0:
        np.save(os.path.join(out_dir, "all.npy"), np.concatenate(shards))
        np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_cover_disjoint_streams(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle as O
    name, S, m = "xoshiro256**", 24, 16
    want = O.bulk_fill(name, "jump", O.seed(name, 42), world * S, m)
    assert (np.load(tmp_path / "all.npy") == want).all()
    assert np.load(tmp_path / "slowest.npy")[0] == 2.5
