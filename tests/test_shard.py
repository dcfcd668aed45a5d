"""Slice sharding across ranks: contiguous cost-balanced ranges (checked against brute force) and the
two-rank path with the gloo backend on CPU (disjoint, covering slice sets; max-over-ranks timing)."""
import itertools
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1905_00934_gb300 import shard


def _brute(costs, parts):
    n = len(costs)
    best = None
    for cuts in itertools.combinations_with_replacement(range(n + 1), parts - 1):
        bounds = (0,) + cuts + (n,)
        worst = max(sum(costs[bounds[k]:bounds[k + 1]]) for k in range(parts))
        best = worst if best is None else min(best, worst)
    return best


@pytest.mark.parametrize("seed", range(20))
def test_partition_is_optimal_and_contiguous(seed):
    import random

    rnd = random.Random(seed)
    n, parts = rnd.randint(1, 9), rnd.randint(1, 4)
    costs = [rnd.choice([1.0, 2.0, 3.5, 7.0, 0.0]) for _ in range(n)]
    r = shard.partition(costs, parts)
    assert len(r) == parts
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(r[k][1] == r[k + 1][0] for k in range(parts - 1))
    assert all(lo <= hi for lo, hi in r)
    assert max(sum(costs[lo:hi]) for lo, hi in r) == pytest.approx(_brute(costs, parts))


def test_equal_slices_split_evenly():
    assert shard.partition([1.0] * 16, 4) == [(0, 4), (4, 8), (8, 12), (12, 16)]
    assert list(shard.rank_slices([1.0] * 16, 2, 4)) == [8, 9, 10, 11]
    assert shard.partition([], 3) == [(0, 0)] * 3
    assert shard.partition([5.0], 3) == [(0, 1), (1, 1), (1, 1)]


def test_slice_cost_grows_with_the_projector_weights():
    a = shard.slice_cost(512, 512, 720, 1024)
    assert shard.slice_cost(1024, 1024, 1440, 2048) == 8 * a
    assert shard.slice_cost(512, 512, 720, 1024, iterations=100) == 100 * a


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = list(shard.rank_slices(costs, rank, ws))
        gathered = [None] * ws
        dist.all_gather_object(gathered, mine)
        slowest = shard.max_over_ranks(10.0 + rank)
        out[rank] = (gathered, slowest)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_disjoint_cover_and_max_time():
    costs = [shard.slice_cost(n, n, v, b) for n, v, b in
             [(256, 360, 512), (1024, 1440, 2048), (512, 720, 1024), (768, 1080, 1536), (256, 360, 512)]]
    ws = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), costs, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        gathered, slowest = res[rank]
        flat = [s for part in gathered for s in part]
        assert sorted(flat) == list(range(len(costs)))          # every slice once
        assert gathered[rank] == list(shard.rank_slices(costs, rank, ws))
        assert slowest == 11.0                                    # max over ranks
    loads = [sum(costs[s] for s in part) for part in res[0][0]]
    assert max(loads) == pytest.approx(_brute(costs, ws))
