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
