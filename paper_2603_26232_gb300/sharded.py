"""One graph's ParaQAOA solve sharded across ranks, one GPU per rank.

The paper's solver pool (Sec. 3.3.1) runs the subgraphs' QAOA circuits on
several GPUs, balanced by subgraph size. The circuits of different parts are
independent, so a rank's part of the work needs nothing from the others:

  1. every rank partitions the same graph (Alg. 1, deterministic host code)
     and computes the same assignment of parts to ranks
     (paraqaoa_shard_plan: longest processing time first on 2^n p);
  2. rank r solves its parts: angle search, final simulation and top-K,
     through the C ABI on its own GPU;
  3. the one exchange: the fixed-size M x K arrays of candidate bitstrings
     and probabilities are summed onto rank 0 (each row is non-zero on
     exactly one rank, so the sum is a gather), and rank 0 merges them into
     the cut of the whole graph (Sec. 3.4).

A part's candidates do not depend on which rank computed them or on which
other parts shared its batches, so the sharded solve returns the cut and
assignment of a single-process solve.

The per-rank solver and the merge are arguments with the CUDA path as their
default; the world-size-2 CPU test substitutes the oracle for them to check
the host logic and the exchange without a GPU.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import _capi


@dataclass
class ShardResult:
    side: np.ndarray | None    # rank 0: assignment of every vertex; None elsewhere
    cut: int | None            # rank 0: CutVal of that assignment
    ranks: np.ndarray          # rank of each part
    loads: np.ndarray          # planned load of each rank (sum of 2^n p over its parts)
    mine: np.ndarray           # ids of the parts this rank solved
    cand: np.ndarray | None    # rank 0: M x K candidate bitstrings of all parts
    cand_p: np.ndarray | None  # rank 0: their probabilities
    times: dict = field(default_factory=dict)


def cuda_part_solver(ctx, cfg):
    """The CUDA path for one rank's parts: angle search, final states, top-K."""
    def solve(part, ids):
        gam, bet, _ = _capi.paraqaoa_angle_search(ctx, part, ids, cfg.p, cfg.grid_points, cfg.adam_steps,
                                                  cfg.lr, cfg.h)
        _, z, pr = _capi.paraqaoa_final_topk(ctx, part, ids, cfg.p, gam, bet, cfg.K)
        return z, pr
    return solve


def cuda_merger(ctx, cfg):
    def merge(G, part, cand):
        return _capi.paraqaoa_merge(ctx, G, part, cand, cfg.K, cfg.L, cfg.beam)
    return merge


def reduce_candidates(dist, ids, z, pr, M: int, K: int, device):
    """Sum the M x K candidate arrays onto rank 0; the rows in ids are this
    rank's, every other row is zero here. Returns the full arrays on rank 0,
    (None, None) on the others."""
    import torch
    zt = torch.zeros((M, K), dtype=torch.int64)
    pt = torch.zeros((M, K), dtype=torch.float32)
    if len(ids):
        zt[torch.as_tensor(ids, dtype=torch.int64)] = torch.as_tensor(np.asarray(z, np.int64))
        pt[torch.as_tensor(ids, dtype=torch.int64)] = torch.as_tensor(np.asarray(pr, np.float32))
    zt, pt = zt.to(device), pt.to(device)
    dist.reduce(zt, dst=0, op=dist.ReduceOp.SUM)
    dist.reduce(pt, dst=0, op=dist.ReduceOp.SUM)
    if dist.get_rank() != 0:
        return None, None
    return zt.cpu().numpy().astype(np.uint32), pt.cpu().numpy()


def solve_sharded(dist, g, cfg, solve_parts, merge, device="cuda") -> ShardResult:
    """Solve graph g with cfg (a SolveConfig) across the ranks of dist.
    solve_parts(part, ids) -> (z, p), each len(ids) x K, solves this rank's
    parts; merge(G, part, cand) -> (side, cut) runs on rank 0."""
    rank, world = dist.get_rank(), dist.get_world_size()
    G = _capi.Graph.of(g)
    t = {}
    t0 = time.perf_counter()
    part = _capi.paraqaoa_partition(G, cfg.M, cfg.mode, cfg.sizes)
    try:
        _, size, _, _ = _capi.paraqaoa_part_info(part)
        M = len(size)
        ranks, loads = _capi.paraqaoa_shard_plan(part, world, cfg.p)
        mine = np.flatnonzero(ranks == rank).astype(np.int32)
        t["plan"] = time.perf_counter() - t0
        if len(mine):
            z, pr = solve_parts(part, mine)
        else:
            z = np.zeros((0, cfg.K), np.uint32)
            pr = np.zeros((0, cfg.K), np.float32)
        t["solve"] = time.perf_counter() - t0 - t["plan"]
        cand, cand_p = reduce_candidates(dist, mine, z, pr, M, cfg.K, device)
        t["exchange"] = time.perf_counter() - t0 - t["plan"] - t["solve"]
        side = cut = None
        if rank == 0:
            side, cut = merge(G, part, cand)
        t["total"] = time.perf_counter() - t0
        return ShardResult(side, cut, ranks, loads, mine, cand, cand_p, t)
    finally:
        _capi.paraqaoa_part_free(part)
