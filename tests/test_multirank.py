"""Replica sharding across ranks (world size 2, gloo, CPU).

Every tile is independent (HiVision Sec. 3.3 splits the pixels evenly), so
ranks holding a replica of the layer and rendering contiguous shards of the
request list must, concatenated, give exactly the single-rank result.  The
tiles are rendered with the oracle here (no GPU on this path); the shard
function is the one bench.py uses.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from workloads import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = gen.gmm_points(20_000, seed=81, k=4)
    reqs = gen.density_tiles(pts, 37, 3, 11, 20, seed=82)
    mine = gen.shard(reqs, rank, world)
    out = oracle.render_points(pts, mine, oracle.MODE_COVERAGE)
    t = torch.from_numpy(out.reshape(-1).copy())
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.numel()]))
    mx = max(int(sz.item()) for sz in sizes)
    padded = torch.zeros(mx, dtype=torch.uint8)
    padded[:t.numel()] = t
    parts = [torch.zeros(mx, dtype=torch.uint8) for _ in sizes]
    dist.all_gather(parts, padded)             # gloo gathers equal sizes: pad, then trim
    parts = [p[:int(sz.item())] for p, sz in zip(parts, sizes)]
    # the slowest rank's time is what a step reports
    tm = torch.tensor([float(rank + 1)])
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    if rank == 0:
        full = torch.cat(parts).numpy().reshape(len(reqs), -1)
        ref = oracle.render_points(pts, reqs, oracle.MODE_COVERAGE)
        np.save(out_path, np.array([np.array_equal(full, ref), tm.item() == world, len(mine)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_concatenate_to_single_rank(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    ok, maxed, n0 = np.load(out)
    assert ok and maxed and n0 == 18


def test_shard_partition():
    from workloads import gen
    rows = np.arange(1001)
    for world in (1, 2, 3, 8):
        parts = [gen.shard(rows, r, world) for r in range(world)]
        assert np.array_equal(np.concatenate(parts), rows)
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def _route_worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2005_12489_gb300 import hv
    from workloads import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = gen.gmm_points(20_000, seed=83, k=4)
    reqs = gen.density_tiles(pts, 41, 3, 11, [12, 20], seed=84)
    route = hv.hv_route_tiles(reqs, world)
    mine = np.nonzero(route == rank)[0]
    out = oracle.render_points(pts, reqs[mine], oracle.MODE_MASK) if len(mine) else np.zeros((0, 8192), np.uint8)
    # every rank sends (request index, tile) for the tiles routed to it
    payload = [None] * world
    dist.all_gather_object(payload, (mine.tolist(), out))
    if rank == 0:
        full = np.zeros((len(reqs), 8192), np.uint8)
        seen = np.zeros(len(reqs), bool)
        for idx, tiles in payload:
            full[idx] = tiles
            seen[idx] = True
        ref = oracle.render_points(pts, reqs, oracle.MODE_MASK)
        np.save(out_path, np.array([np.array_equal(full, ref), seen.all(), min(len(p[0]) for p in payload)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_router_partitions_and_reassembles(tmp_path):
    """The tile router (hv_route_tiles) splits a batch between two replica
    ranks; the tiles each renders, put back by request index, are the
    single-rank result."""
    import torch.multiprocessing as mp
    from paper_2005_12489_gb300 import build
    build.build()
    out = str(tmp_path / "route.npy")
    mp.start_processes(_route_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    ok, covered, n_min = np.load(out)
    assert ok and covered and n_min > 0


def test_router_properties():
    from paper_2005_12489_gb300 import build, hv
    from workloads import gen
    build.build()
    pts = gen.gmm_points(100_000, seed=85, k=16)
    reqs = hv.make_requests(gen.density_tiles(pts, 20_000, 0, 19, 16, seed=86))
    for n in (1, 2, 3, 8):
        r = hv.hv_route_tiles(reqs, n)
        assert r.max() < n and np.array_equal(r, hv.hv_route_tiles(reqs, n))
    # the same tile goes to the same rank whatever its radius, mode or order
    other = reqs.copy()
    other["r16"], other["mode"] = 900, 2
    assert np.array_equal(hv.hv_route_tiles(other[::-1], 8)[::-1], hv.hv_route_tiles(reqs, 8))
    # distinct tiles spread evenly
    key = reqs["z"].astype(np.int64) * (1 << 40) + reqs["x"].astype(np.int64) * (1 << 20) + reqs["y"]
    _, first = np.unique(key, return_index=True)
    counts = np.bincount(hv.hv_route_tiles(reqs[first], 8), minlength=8)
    assert counts.min() > 0.85 * counts.mean()
