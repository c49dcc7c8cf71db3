"""The N > 1 path on the host: two gloo ranks on CPU (no GPU).

Cells are independent, so ranks shard them with no collective on the data path; the only
collectives are the benchmark's barrier and its max/sum of scalars.  These tests run those on two
processes and check the cell partition."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_21278_b300.shard import cell_cost, partition_cells

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank_main(rank, world, port, counts, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench_module()
        ws, r = b._dist()
        assert (ws, r) == (world, rank)
        b._barrier(ws)
        mx = b._max_over_ranks(float(rank + 1), ws)
        sm = b._sum_over_ranks(float(10 * (rank + 1)), ws)
        mine = partition_cells(counts, 64, world)[rank]
        sizes = [None] * world
        dist.all_gather_object(sizes, mine.tolist())
        out[rank] = (mx, sm, sizes)
    finally:
        dist.destroy_process_group()


def _cell_keys(wl):
    """(sample count, first sample's x, y) of every cell: identifies a cell of the seeded replicas."""
    off = wl.offsets.tolist()
    return sorted((off[j + 1] - off[j], float(wl.x[off[j]]), float(wl.y[off[j]])) for j in range(wl.n_cells)
                  if off[j + 1] > off[j])


def _slice_main(rank, world, port, out):
    import argparse
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench_module()
        args = argparse.Namespace(workload="tri20480_p64", cells=40, q_scale=0.02, max_q=None, tc_max_points=None,
                                  frame="centroid")
        wl = b._rank_workload(args, world, rank, "cpu")
        keys = [None] * world
        dist.all_gather_object(keys, (wl.n_cells, wl.n_points, _cell_keys(wl)))
        out[rank] = keys
        # the gradient path's only collective: one binary64 scalar summed over the ranks
        out[f"L{rank}"] = b._sum_over_ranks(float(rank + 0.5), world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_one_seeded_batch():
    """bench.py's job is one seeded batch of `world` replicas split by LPT: the union of the two ranks'
    cells is exactly the set of cells of the replicas, no cell twice, and the loss reduction adds the
    ranks' scalars."""
    import synth
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_slice_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    per_rank = out[0]
    assert per_rank == out[1]
    union = sorted(k for r in range(world) for k in per_rank[r][2])
    expect = sorted(k for s in range(world)
                    for k in _cell_keys(synth.make("tri20480_p64", seed=s, n_cells=40, q_scale=0.02)))
    assert union == expect
    assert sum(per_rank[r][0] for r in range(world)) == 2 * 40
    assert out["L0"] == out["L1"] == 2.0


def test_two_gloo_ranks_reduce_and_agree_on_the_partition():
    world = 2
    counts = np.random.default_rng(0).integers(500, 20000, size=301)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), counts, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        mx, sm, parts = out[r]
        assert mx == 2.0 and sm == 30.0
        assert parts == out[0][2]          # every rank computes the same split
    allc = sorted(sum(out[0][2], []))
    assert allc == list(range(len(counts)))   # each cell on exactly one rank


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_covers_cells_once_and_balances(world):
    counts = np.random.default_rng(world).lognormal(np.log(4000), 0.55, size=2000).astype(int)
    parts = partition_cells(counts, 64, world)
    cat = np.sort(np.concatenate(parts))
    assert np.array_equal(cat, np.arange(len(counts)))
    cost = cell_cost(counts, 64)
    loads = np.array([cost[p].sum() for p in parts])
    # LPT bound: no rank exceeds the mean by more than the largest single cell
    assert loads.max() - loads.mean() <= cost.max() + 1e-6


def test_partition_edge_cases():
    assert [p.tolist() for p in partition_cells([], 64, 2)] == [[], []]
    assert [p.tolist() for p in partition_cells([5], 64, 3)] == [[0], [], []]
    with pytest.raises(ValueError):
        partition_cells([1, 2], 64, 0)
