"""GB300-native ParaQAOA hot path (arXiv 2603.26232).

The CUDA library (libparaqaoa.so, built from csrc/ for sm_103a) does the
work; this package only binds its C ABI (``_capi``, same names as the header
include/paraqaoa.h) and strings the calls of one ParaQAOA solve together.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import _capi
from ._capi import *  # noqa: F401,F403  (the C-ABI functions and constants)
from ._capi import Graph, ParaQAOAError


def build(force: bool = False) -> str:
    from .native_build import build as _b
    return _b(force=force)


@dataclass
class SolveConfig:
    M: int                   # number of parts (Sec. 3.2)
    K: int = 4               # top-K per part (Sec. 3.3.2)
    p: int = 1               # QAOA depth
    grid_points: int = 16    # p = 1 grid
    adam_steps: int = 0      # Adam steps per depth (0: grid only)
    lr: float = 0.02
    h: float = 1e-3
    L: int = 1               # merge starting level (exhaustive merge)
    beam: int = 0            # 0: exhaustive merge; > 0: beam width
    mode: int = _capi.PART_BALANCED
    sizes: np.ndarray | None = None
    mlp: object = None       # trained angle network (paraqaoa_mlp) of depth p: learned form
    fallback_steps: int = 32  # Adam steps of the plain form for parts the judge rejects
    judge_tol: float = 0.0   # judge tolerance (fraction of W) before a part falls back


@dataclass
class SolveResult:
    side: np.ndarray
    cut: int
    gamma: np.ndarray
    beta: np.ndarray
    expect: np.ndarray
    cand: np.ndarray
    cand_p: np.ndarray
    times: dict = field(default_factory=dict)


class Solver:
    """One CUDA context and the full ParaQAOA pipeline on it:
    partition -> angle search -> final simulation -> top-K -> merge."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, halved: bool = False):
        self.ctx = _capi.paraqaoa_create(device, hbm_budget)
        if halved:  # parts of >= 16 vertices simulated on half their state (psi_z = psi_(not z))
            _capi.paraqaoa_set_halved(self.ctx, True)

    def close(self):
        if self.ctx:
            _capi.paraqaoa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, g, cfg: SolveConfig) -> SolveResult:
        G = Graph.of(g)
        t = {}
        t0 = time.perf_counter()
        part = _capi.paraqaoa_partition(G, cfg.M, cfg.mode, cfg.sizes)
        try:
            _, size, _, _ = _capi.paraqaoa_part_info(part)
            ids = np.arange(len(size), dtype=np.int32)
            _capi.paraqaoa_part_upload(self.ctx, part)
            t["partition"] = time.perf_counter() - t0
            fallback = None
            if cfg.mlp is not None:
                gam, bet, val, fallback = _capi.paraqaoa_solve_learned(self.ctx, part, ids, cfg.mlp, cfg.p,
                                                                       cfg.fallback_steps, cfg.judge_tol)
            else:
                gam, bet, val = _capi.paraqaoa_angle_search(self.ctx, part, ids, cfg.p, cfg.grid_points,
                                                            cfg.adam_steps, cfg.lr, cfg.h)
            t["angles"] = time.perf_counter() - t0 - t["partition"]
            ex, cand, cand_p = _capi.paraqaoa_final_topk(self.ctx, part, ids, cfg.p, gam, bet, cfg.K)
            t["final"] = time.perf_counter() - t0 - t["partition"] - t["angles"]
            side, cut = _capi.paraqaoa_merge(self.ctx, G, part, cand, cfg.K, cfg.L, cfg.beam)
            t["merge"] = time.perf_counter() - t0 - t["partition"] - t["angles"] - t["final"]
            t["total"] = time.perf_counter() - t0
            res = SolveResult(side, cut, gam, bet, ex, cand, cand_p, t)
            res.fallback = fallback
            return res
        finally:
            _capi.paraqaoa_part_free(part)
