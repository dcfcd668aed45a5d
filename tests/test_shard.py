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


def _run_sum(a):
    t = 0.0
    for c in a:
        t += c
    return t


def test_partition_is_exact_where_run_sums_round():
    # a candidate cap formed as a difference of prefix sums can fall one ulp below the running sum
    # that the fill compares with; the partition must still reach the optimum (here 4e6 + the tail)
    costs = [4e6, 4e6, 0.0, 3.5, 6.074379962852603, 7.0, 0.0, 0.0, 9.391491627785106]
    r = shard.partition(costs, 2)
    assert r == [(0, 1), (1, 9)]
    # one part: the whole batch, even where Python's compensated sum() differs from the running total
    costs = [0.0, 4e6, 7.0, 2.0, 3.5, 1.7467058960990223, 4e6, 3.5, 7.0, 2e6, 2.0, 9.206200381334538, 2.0] * 3
    assert shard.partition(costs, 1) == [(0, len(costs))]


def test_partition_of_the_largest_batch_is_fast_and_balanced():
    import random
    import time

    rnd = random.Random(3)
    costs = [rnd.uniform(1.0, 100.0) for _ in range(4096)]  # the solver's largest batch
    t0 = time.perf_counter()
    r = shard.partition(costs, 8)
    assert time.perf_counter() - t0 < 2.0
    assert len(r) == 8 and r[0][0] == 0 and r[-1][1] == 4096
    worst = max(_run_sum(costs[lo:hi]) for lo, hi in r)
    assert worst <= _run_sum(costs) / 8 + max(costs)  # within one slice of the even share
