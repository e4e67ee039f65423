"""ParaQAOA CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain double-precision reference for the CUDA path. Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it; the
product package never imports it. The numerics live in ``paraqaoa_oracle.c``
(compiled with gcc by :func:`build`); this module marshals arguments and holds
the angle-search drivers, whose scalar arithmetic is FP64 numpy.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: the p=1 closed form, dense matrix exponentials, brute force, symmetry
laws and the paper's worked examples.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paraqaoa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, ESEARCH = 0, -1, -4, -5


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.or_cutval.argtypes = [i32, P, P, P, P]
        L.or_cutval.restype = i64
        L.or_cut_table.argtypes = [i32, i64, P, P, P, P]
        L.or_partition.argtypes = [i32, i32, i32, P, P, P]
        L.or_get_subgraph.argtypes = [i32, P, P, P, i32, i32, P, P, P]
        L.or_get_subgraph.restype = i64
        L.or_simulate.argtypes = [i32, i64, P, P, P, i32, P, P, P]
        L.or_expect_state.argtypes = [i32, P, P]
        L.or_expect_state.restype = f64
        L.or_expect_batch.argtypes = [i32, P, P, P, P, P, i32, P, i32, P, P, P]
        L.or_topk.argtypes = [i32, P, i32, i32, P, P]
        L.or_bruteforce_maxcut.argtypes = [i32, i64, P, P, P, P]
        L.or_bruteforce_maxcut.restype = i64
        L.or_merge_exhaustive.argtypes = [i32, P, P, P, i32, P, P, P, i32, i32, P, P, P]
        L.or_merge_beam.argtypes = [i32, P, P, P, i32, P, P, P, i32, i64, P, P]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------- graphs
def cutval(g, side) -> int:
    """Sec. 2.1 CutVal of a full-graph assignment."""
    s = _c(side, np.uint8)
    return int(lib().or_cutval(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(s)))


@dataclass
class Subgraph:
    first: int  # global index of local vertex 0
    n: int
    eu: np.ndarray
    ev: np.ndarray
    ew: np.ndarray

    @property
    def total_weight(self) -> int:
        return int(self.ew.astype(np.int64).sum())


def partition(num_vertices: int, M: int, mode: int = 0, sizes=None):
    """Alg. 1 (modes: 0 balanced reading, 1 literal, 2 explicit sizes) ->
    (first vertex, size) arrays."""
    first = np.zeros(M, np.int32)
    size = np.zeros(M, np.int32)
    sz = _c(sizes if sizes is not None else np.zeros(M), np.int32)
    rc = lib().or_partition(num_vertices, M, mode, _p(sz), _p(first), _p(size))
    if rc != OK:
        raise ValueError(f"partition rejected (rc={rc})")
    return first, size


def get_subgraph(g, first: int, size: int) -> Subgraph:
    """Alg. 1 GetSubgraph: the induced edges of V_i = [first, first+size)."""
    L = lib()
    cnt = L.or_get_subgraph(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), first, size, None, None, None)
    eu = np.zeros(cnt, np.int32)
    ev = np.zeros(cnt, np.int32)
    ew = np.zeros(cnt, np.int32)
    L.or_get_subgraph(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), first, size, _p(eu), _p(ev), _p(ew))
    return Subgraph(int(first), int(size), eu, ev, ew)


def subgraphs(g, M: int, mode: int = 0, sizes=None) -> list[Subgraph]:
    first, size = partition(g.n, M, mode, sizes)
    return [get_subgraph(g, int(f), int(s)) for f, s in zip(first, size)]


def inter_edges(g, subs: list[Subgraph]):
    """E_inter (Sec. 3.4.1): edges of G not inside any part, as (u, v, w), u < v."""
    inside = set()
    for s in subs:
        for a, b in zip(s.eu, s.ev):
            inside.add((s.first + int(a), s.first + int(b)))
    keep = [(int(a), int(b), int(c)) for a, b, c in zip(g.eu, g.ev, g.ew) if (int(a), int(b)) not in inside]
    return keep


# ---------------------------------------------------------------- simulation
def cut_table(s: Subgraph) -> np.ndarray:
    out = np.zeros(1 << s.n, np.int64)
    lib().or_cut_table(s.n, len(s.eu), _p(s.eu), _p(s.ev), _p(s.ew), _p(out))
    return out


def simulate(s: Subgraph, gamma, beta) -> np.ndarray:
    """Sec. 2.2: the complex128 QAOA state after p = len(gamma) layers."""
    g = _c(np.atleast_1d(gamma), np.float64)
    b = _c(np.atleast_1d(beta), np.float64)
    assert g.size == b.size
    st = np.zeros(2 << s.n, np.float64)
    rc = lib().or_simulate(s.n, len(s.eu), _p(s.eu), _p(s.ev), _p(s.ew), g.size, _p(g), _p(b), _p(st))
    if rc != OK:
        raise ValueError(f"simulate rejected (rc={rc})")
    return st.view(np.complex128)


def expect_state(s: Subgraph, state: np.ndarray, cut=None) -> float:
    cut = cut_table(s) if cut is None else _c(cut, np.int64)
    st = _c(state, np.complex128).view(np.float64)
    return float(lib().or_expect_state(s.n, _p(st), _p(cut)))


class Batch:
    """Flattened edge lists of several subgraphs for the batched calls."""

    def __init__(self, subs: list[Subgraph]):
        self.subs = subs
        self.nq = np.array([s.n for s in subs], np.int32)
        self.edge_off = np.zeros(len(subs) + 1, np.int64)
        np.cumsum([len(s.eu) for s in subs], out=self.edge_off[1:])
        cat = lambda k: (np.concatenate([getattr(s, k) for s in subs]).astype(np.int32)
                         if self.edge_off[-1] else np.zeros(1, np.int32))
        self.eu, self.ev, self.ew = cat("eu"), cat("ev"), cat("ew")


def expect_batch(batch: Batch, sub_idx, gamma, beta) -> np.ndarray:
    """<C> for instances (sub_idx[i], gamma[i,:], beta[i,:])."""
    sub_idx = _c(sub_idx, np.int32)
    gamma = _c(gamma, np.float64).reshape(len(sub_idx), -1)
    beta = _c(beta, np.float64).reshape(len(sub_idx), -1)
    p = gamma.shape[1]
    out = np.zeros(len(sub_idx), np.float64)
    rc = lib().or_expect_batch(len(batch.subs), _p(batch.nq), _p(batch.edge_off), _p(batch.eu),
                               _p(batch.ev), _p(batch.ew), len(sub_idx), _p(sub_idx), p,
                               _p(gamma), _p(beta), _p(out))
    if rc != OK:
        raise ValueError(f"expect_batch rejected (rc={rc})")
    return out


def topk(n: int, state: np.ndarray, K: int, canonical: bool = True):
    """Sec. 3.3.2: K most probable z, key (probability desc, z asc)."""
    st = _c(state, np.complex128).view(np.float64)
    z = np.zeros(K, np.uint32)
    pr = np.zeros(K, np.float64)
    rc = lib().or_topk(n, _p(st), K, 1 if canonical else 0, _p(z), _p(pr))
    if rc != OK:
        raise ValueError(f"topk rejected (rc={rc})")
    return z, pr


def bruteforce_maxcut(s: Subgraph):
    bz = np.zeros(1, np.uint32)
    best = lib().or_bruteforce_maxcut(s.n, len(s.eu), _p(s.eu), _p(s.ev), _p(s.ew), _p(bz))
    return int(best), int(bz[0])


# ---------------------------------------------------------------- merge
def merge_exhaustive(g, first, size, cand, K: int, L: int = 1):
    first, size = _c(first, np.int32), _c(size, np.int32)
    cand = _c(cand, np.uint32)
    side = np.zeros(g.n, np.uint8)
    cut = np.zeros(1, np.int64)
    leaves = np.zeros(1, np.int64)
    rc = lib().or_merge_exhaustive(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), len(first), _p(first),
                                   _p(size), _p(cand), K, L, _p(side), _p(cut), _p(leaves))
    if rc != OK:
        raise ValueError(f"merge rejected (rc={rc})")
    return side, int(cut[0]), int(leaves[0])


def merge_beam(g, first, size, cand, K: int, beam: int):
    first, size = _c(first, np.int32), _c(size, np.int32)
    cand = _c(cand, np.uint32)
    side = np.zeros(g.n, np.uint8)
    cut = np.zeros(1, np.int64)
    rc = lib().or_merge_beam(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), len(first), _p(first),
                             _p(size), _p(cand), K, int(beam), _p(side), _p(cut))
    if rc != OK:
        raise ValueError(f"merge rejected (rc={rc})")
    return side, int(cut[0])


# ---------------------------------------------------------------- angle search
# The paper leaves the optimiser open (Sec. 2.2 names gradient descent or
# evolutionary strategies; Sec. 2.2 also notes initialisation matters). The
# reading used here: a fixed grid for p = 1 (gamma axis divided by the mean
# edge weight in the plain form), INTERP initialisation for p > 1
# (Zhou et al., PRX 10, 021067, 2020), then a fixed number of Adam steps on
# -<C>/W with central-difference gradients; all scalars FP64.

def grid_points(points: int = 16):
    a = np.arange(points, dtype=np.float64)
    return np.repeat(np.pi * a / points, points), np.tile((np.pi / 2) * a / points, points)


def grid_scale(s: Subgraph) -> float:
    """The plain form's gamma-axis divisor of one subgraph: its mean edge
    weight, at least 1 (1 for an edgeless subgraph)."""
    return max(1.0, float(np.mean(s.ew))) if len(s.ew) else 1.0


def grid_search(batch: Batch, points: int = 16, weight_scaled: bool = False):
    """For every subgraph: <C> at every grid point and the first maximum in
    row-major (gamma index, beta index) order. Grid gamma_a = pi a / points,
    beta_b = (pi/2) b / points; with weight_scaled (the plain form's grid)
    subgraph i's gamma axis is divided by grid_scale: gamma_a = pi a /
    (points s_i)."""
    g, b = grid_points(points)
    S = len(batch.subs)
    G = g.size
    sc = np.array([grid_scale(s) if weight_scaled else 1.0 for s in batch.subs])
    gam = (g[None, :] / sc[:, None]).reshape(-1)
    sub_idx = np.repeat(np.arange(S, dtype=np.int32), G)
    vals = expect_batch(batch, sub_idx, gam, np.tile(b, S)).reshape(S, G)
    arg = np.argmax(vals, axis=1)  # numpy argmax returns the first maximum
    return vals, arg, g[arg] / sc, b[arg]


def interp(gamma: np.ndarray, beta: np.ndarray):
    """INTERP: depth-p angles -> depth-(p+1) angles (Zhou et al. 2020)."""
    p = gamma.shape[-1]

    def one(x):
        x0 = np.concatenate([np.zeros(x.shape[:-1] + (1,)), x, np.zeros(x.shape[:-1] + (1,))], axis=-1)
        out = np.zeros(x.shape[:-1] + (p + 1,))
        for i in range(1, p + 2):
            out[..., i - 1] = ((i - 1) / p) * x0[..., i - 1] + ((p - i + 1) / p) * x0[..., i]
        return out

    return one(gamma), one(beta)


def canonicalize(gamma: np.ndarray, beta: np.ndarray):
    """Fold angles into one fundamental domain: (gamma, beta) -> (-gamma,
    -beta) leaves every probability unchanged, gamma has period 2 pi for
    integer cut values and beta period pi/2; result gamma_1 in [0, pi],
    other gammas in (-pi, pi], betas in (-pi/4, pi/4]."""
    g = np.array(gamma, dtype=np.float64, copy=True)
    b = np.array(beta, dtype=np.float64, copy=True)
    g = np.mod(g + np.pi, 2 * np.pi) - np.pi  # (-pi, pi] up to the endpoint
    g = np.where(g <= -np.pi, g + 2 * np.pi, g)
    flip = g[..., :1] < 0
    g = np.where(flip, -g, g)
    b = np.where(flip, -b, b)
    g = np.mod(g + np.pi, 2 * np.pi) - np.pi
    g = np.where(g <= -np.pi, g + 2 * np.pi, g)
    b = np.mod(b + np.pi / 4, np.pi / 2) - np.pi / 4
    b = np.where(b <= -np.pi / 4, b + np.pi / 2, b)
    return g, b


@dataclass
class AdamConfig:
    steps: int = 32
    lr: float = 0.02
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    h: float = 1e-3


def adam_optimize(batch: Batch, gamma0, beta0, cfg: AdamConfig = AdamConfig(), expect_fn=None):
    """Fixed-iteration Adam on f = -<C>/W for every subgraph at once.
    Each step evaluates f at theta +- h e_k for all 2p angles (central
    differences), then takes one Adam step. Returns the final angles and
    <C> there. ``expect_fn(sub_idx, gamma, beta)`` defaults to the oracle."""
    expect_fn = expect_fn or (lambda si, g, b: expect_batch(batch, si, g, b))
    S = len(batch.subs)
    p = np.asarray(gamma0).shape[-1]
    W = np.array([max(s.total_weight, 1) for s in batch.subs], np.float64)
    theta = np.concatenate([np.asarray(gamma0, np.float64).reshape(S, p),
                            np.asarray(beta0, np.float64).reshape(S, p)], axis=1)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    sub_idx = np.repeat(np.arange(S, dtype=np.int32), 4 * p)
    for t in range(1, cfg.steps + 1):
        shifts = np.zeros((S, 4 * p, 2 * p))
        for k in range(2 * p):
            shifts[:, 2 * k, k] = cfg.h
            shifts[:, 2 * k + 1, k] = -cfg.h
        th = (theta[:, None, :] + shifts).reshape(S * 4 * p, 2 * p)
        f = -expect_fn(sub_idx, th[:, :p], th[:, p:]).reshape(S, 2 * p, 2) / W[:, None, None]
        grad = (f[:, :, 0] - f[:, :, 1]) / (2 * cfg.h)
        m = cfg.beta1 * m + (1 - cfg.beta1) * grad
        v = cfg.beta2 * v + (1 - cfg.beta2) * grad * grad
        mh = m / (1 - cfg.beta1 ** t)
        vh = v / (1 - cfg.beta2 ** t)
        theta = theta - cfg.lr * mh / (np.sqrt(vh) + cfg.eps)
    g, b = theta[:, :p], theta[:, p:]
    final = expect_fn(np.arange(S, dtype=np.int32), g, b)
    return g, b, final
