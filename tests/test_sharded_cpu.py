"""One graph's solve sharded across ranks (paper_2603_26232_gb300.sharded),
checked on CPU: the longest-processing-time plan against a hand-worked case
and Graham's bound (brute force over every assignment of tiny cases), and
two gloo ranks whose sharded solve returns the single-process cut and
assignment bit for bit. The per-part solver and the merge are the FP64
oracle here (no GPU); the plan, the candidate exchange and the bookkeeping
are the product's."""
import itertools
import os
import socket

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.fixture(scope="module")
def capi():
    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi
    _capi.load()
    return _capi


def _part_of_sizes(capi, sizes, seed=0, p_edge=0.3, wmax=5):
    nv = int(sum(sizes) - (len(sizes) - 1))
    g = synth.erdos_renyi(nv, p_edge, seed, wmax=wmax)
    return g, capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)


def test_shard_plan_hand_worked(capi):
    # costs 2^n p at p = 1: 8, 32, 16, 32, 4. By cost descending (ties by
    # index): parts 1, 3, 2, 0, 4. Two ranks: 1 -> r0 (32), 3 -> r1 (32),
    # 2 -> r0 (tie, lowest rank; 48), 0 -> r1 (40), 4 -> r1 (44).
    # Three ranks: 1 -> r0, 3 -> r1, 2 -> r2 (16), 0 -> r2 (24), 4 -> r2 (28).
    _, part = _part_of_sizes(capi, [3, 5, 4, 5, 2])
    try:
        r2, l2 = capi.paraqaoa_shard_plan(part, 2, 1)
        assert r2.tolist() == [1, 0, 0, 1, 1] and l2.tolist() == [48.0, 44.0]
        r3, l3 = capi.paraqaoa_shard_plan(part, 3, 1)
        assert r3.tolist() == [2, 0, 2, 1, 2] and l3.tolist() == [32.0, 32.0, 28.0]
        # p scales every cost; evals weights each part
        r, l = capi.paraqaoa_shard_plan(part, 2, 3)
        assert r.tolist() == r2.tolist() and l.tolist() == [144.0, 132.0]
        # costs 0, 32, 16, 32, 400: part 4 alone on r0, the rest on r1
        r, l = capi.paraqaoa_shard_plan(part, 2, 1, [0, 1, 1, 1, 100])
        assert r.tolist() == [1, 1, 1, 1, 0] and l.tolist() == [400.0, 80.0]
        # one rank takes everything; more ranks than parts leaves some idle
        r1, l1 = capi.paraqaoa_shard_plan(part, 1, 1)
        assert r1.tolist() == [0] * 5 and l1.tolist() == [92.0]
        r8, l8 = capi.paraqaoa_shard_plan(part, 8, 1)
        assert sorted(r8.tolist()) == [0, 1, 2, 3, 4] and l8.sum() == 92.0
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_shard_plan(part, 0, 1)
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("seed", range(6))
def test_shard_plan_within_graham_bound(capi, seed):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(2, 9, int(rng.integers(3, 8))).tolist()
    world = int(rng.integers(2, 4))
    _, part = _part_of_sizes(capi, sizes, seed)
    try:
        ranks, loads = capi.paraqaoa_shard_plan(part, world, 1)
    finally:
        capi.paraqaoa_part_free(part)
    cost = [2.0 ** s for s in sizes]
    # the plan's loads are its assignment's loads
    assert np.allclose(loads, [sum(c for c, r in zip(cost, ranks) if r == k) for k in range(world)])
    best = min(max(sum(c for c, r in zip(cost, a) if r == k) for k in range(world))
               for a in itertools.product(range(world), repeat=len(sizes)))
    assert loads.max() <= (4 / 3 - 1 / (3 * world)) * best + 1e-9


# ---------------------------------------------------------------- two ranks
SIZES, K, GRID = [12, 8, 10, 9, 11, 7], 4, 8


def _oracle_part_solver(orc, g, first, size):
    """FP64 oracle per part: the p = 1 grid's best point, then the top-K of
    the state there (canonical half)."""
    subs = [orc.get_subgraph(g, int(f), int(s)) for f, s in zip(first, size)]

    def solve(part, ids):
        batch = orc.Batch([subs[i] for i in ids])
        _, _, gam, bet = orc.grid_search(batch, GRID)
        z = np.zeros((len(ids), K), np.uint32)
        pr = np.zeros((len(ids), K), np.float32)
        for j, i in enumerate(ids):
            st = orc.simulate(subs[i], [gam[j]], [bet[j]])
            z[j], pr[j] = orc.topk(subs[i].n, st, K)
        return z, pr
    return solve


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        import paper_2603_26232_gb300 as pkg
        from paper_2603_26232_gb300 import sharded
        nv = int(sum(SIZES) - (len(SIZES) - 1))
        g = synth.erdos_renyi(nv, 0.35, 5, wmax=5)
        first, size = orc.partition(nv, len(SIZES), 2, SIZES)
        cfg = pkg.SolveConfig(M=len(SIZES), K=K, p=1, mode=2, sizes=np.array(SIZES, np.int32))
        solve = _oracle_part_solver(orc, g, first, size)
        merge = lambda G, part, cand: orc.merge_exhaustive(g, first, size, cand, K, 1)[:2]  # noqa: E731
        r = sharded.solve_sharded(dist, g, cfg, solve, merge, device="cpu")
        out[rank] = (r.mine.tolist(), r.ranks.tolist(), None if r.side is None else r.side.tolist(), r.cut,
                     None if r.cand is None else r.cand.tolist())
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_single_process(capi, orc):
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    mine0, ranks, side, cut, cand = res[0]
    mine1 = res[1][0]
    # the plan splits the parts between the ranks, both ranks agree on it
    assert sorted(mine0 + mine1) == list(range(len(SIZES))) and res[1][1] == ranks
    assert mine0 and mine1 and res[1][2] is None
    # single process: every part on one rank, then the same merge
    nv = int(sum(SIZES) - (len(SIZES) - 1))
    g = synth.erdos_renyi(nv, 0.35, 5, wmax=5)
    first, size = orc.partition(nv, len(SIZES), 2, SIZES)
    z, _ = _oracle_part_solver(orc, g, first, size)(None, np.arange(len(SIZES)))
    assert np.array_equal(np.array(cand, np.uint32), z)
    side1, cut1, _ = orc.merge_exhaustive(g, first, size, z, K, 1)
    assert cut == cut1 and side == side1.tolist()
    assert orc.cutval(g, np.array(side, np.uint8)) == cut
