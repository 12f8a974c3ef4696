"""Partition of independent strings across ranks (host logic of the multi-GPU strings
run): a partition of every index, the list-scheduling load bound, the 4/3 bound of
longest-processing-time-first against brute-force optima on tiny inputs, and two gloo
ranks that build their own strings and together hold the whole model."""
import itertools
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2102_11026_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _string_costs(n=320, seed=4):
    rs, vs = synth.string_shapes(n, seed)
    return [shard.string_cost(synth.string_widths(r, V)) for r, V in zip(rs, vs)]


def test_string_cost_is_weights_times_columns():
    w = [3, 32, 64, 30]
    assert shard.string_cost(w) == (3 * 32 + 32 * 64 + 64 * 30) * (4 * 3 + 4)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7, 8])
def test_partition_and_list_scheduling_bound(world):
    costs = _string_costs()
    parts = shard.shard_by_cost(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    assert all(p == sorted(p) for p in parts)
    loads = [sum(costs[i] for i in p) for p in parts]
    total, cmax = sum(costs), max(costs)
    assert max(loads) <= total / world + (1 - 1 / world) * cmax
    # 320 strings over 8 ranks: balanced to within one string's cost
    assert max(loads) - min(loads) <= cmax
    assert shard.shard_by_cost(costs, world) == parts          # same on every rank
    if world == 1:
        assert parts == [list(range(len(costs)))]


def test_longest_first_within_four_thirds_of_optimum():
    rng = np.random.default_rng(11)
    for trial in range(40):
        n, m = int(rng.integers(2, 9)), int(rng.integers(2, 4))
        costs = [int(c) for c in rng.integers(1, 50, n)]
        best = min(max(sum(c for c, a in zip(costs, asg) if a == k) for k in range(m))
                   for asg in itertools.product(range(m), repeat=n))
        loads = [sum(costs[i] for i in p) for p in shard.shard_by_cost(costs, m)]
        assert max(loads) <= (4 / 3 - 1 / (3 * m)) * best + 1e-9, (costs, m, loads, best)


def test_edge_cases():
    assert shard.shard_by_cost([], 3) == [[], [], []]
    assert shard.shard_by_cost([5], 2) == [[0], []]
    assert shard.shard_by_cost([2, 2, 2, 2], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.shard_by_cost([1], 0)


def test_subset_of_strings_equals_full_list():
    full = synth.strings(5, seed=9, v_range=(200, 260))
    sub = synth.strings(5, seed=9, v_range=(200, 260), only=[4, 1])
    for a, b in ((full[4], sub[0]), (full[1], sub[1])):
        assert a.dec.widths == b.dec.widths
        assert all(np.array_equal(x, y) for x, y in zip(a.dec.W, b.dec.W))
        assert np.array_equal(a.mesh.X, b.mesh.X) and np.array_equal(a.cub_w, b.cub_w)
        assert np.array_equal(a.state.qbar, b.state.qbar)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_2102_11026_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 12
        rs, vs = synth.string_shapes(n, 4, v_range=(200, 400))
        costs = [shard.string_cost(synth.string_widths(r, V)) for r, V in zip(rs, vs)]
        mine = shard.shard_by_cost(costs, world)[rank]
        wls = synth.strings(n, v_range=(200, 400), only=mine)
        held = [(i, wl.dec.widths[0], wl.mesh.n_vert) for i, wl in zip(mine, wls)]
        got = [None] * world
        dist.all_gather_object(got, held)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_ranks_hold_every_string_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res[0] == res[1]
    held = sorted(x for part in res[0] for x in part)
    rs, vs = synth.string_shapes(12, 4, v_range=(200, 400))
    assert [i for i, _, _ in held] == list(range(12))
    assert [r for _, r, _ in held] == rs
    assert [nv for _, _, nv in held] == vs
