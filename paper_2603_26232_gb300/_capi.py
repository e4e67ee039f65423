"""ctypes binding of libparaqaoa.so: one Python function per C entry point,
same names, argument marshalling only (numpy arrays in, numpy arrays out).

Every computation runs in the CUDA library. There is no CPU fallback: if
the shared library is missing or cannot be loaded, importing this module's
functions raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparaqaoa.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "paraqaoa.h")

OK = 0
E_INVAL, E_TOO_MANY_QUBITS, E_ADMISSION, E_NOMEM = -1, -2, -3, -4
E_SEARCH_TOO_LARGE, E_CUDA, E_TIMEOUT, E_NO_RESULT = -5, -6, -7, -8
E_SCRATCH_LIMIT = -9
PART_BALANCED, PART_ALG1_LITERAL, PART_SIZES = 0, 1, 2
SIM_EXPECT, SIM_KEEP_STATE, SIM_HALVED = 0x1, 0x2, 0x4
SCHED_SPLIT, SCHED_HIGH_FIRST = 0x1, 0x2
TOPK_CANONICAL, TOPK_RAW = 0x0, 0x1
KCLASS_LAYER_PASS, KCLASS_SMEM_SIM, KCLASS_TOPK, KCLASS_MERGE, KCLASS_OTHER, KCLASS_TC_MIXER = range(6)
TC_BF16, TC_FP16 = 0, 1
MAX_TOPK = 32
MAX_SUBGRAPH_WEIGHT = 4095


class ParaQAOAError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("w", ctypes.c_void_p)]


_lib = None
P = ctypes.c_void_p
_SIGS = {
    "paraqaoa_create": ([ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
    "paraqaoa_destroy": ([P], None),
    "paraqaoa_set_stream": ([P, P], ctypes.c_int),
    "paraqaoa_partition": ([P, ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(P)], ctypes.c_int),
    "paraqaoa_part_free": ([P], None),
    "paraqaoa_part_info": ([P, P, P, P, P, P], ctypes.c_int),
    "paraqaoa_part_edges": ([P, ctypes.c_int32, P, P, P], ctypes.c_int),
    "paraqaoa_shard_plan": ([P, ctypes.c_int32, ctypes.c_int32, P, P, P], ctypes.c_int),
    "paraqaoa_part_upload": ([P, P, ctypes.c_int32], ctypes.c_int),
    "paraqaoa_cut_table": ([P, P, ctypes.c_int32, P], ctypes.c_int),
    "paraqaoa_simulate_batch": ([P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_uint32], ctypes.c_int),
    "paraqaoa_expect": ([P, ctypes.c_int32, P], ctypes.c_int),
    "paraqaoa_topk": ([P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_uint32], ctypes.c_int),
    "paraqaoa_state": ([P, ctypes.c_int32, P], ctypes.c_int),
    "paraqaoa_merge": ([P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, P], ctypes.c_int),
    "paraqaoa_grid_search": ([P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P], ctypes.c_int),
    "paraqaoa_optimize": ([P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                           ctypes.c_double, P, P, P], ctypes.c_int),
    "paraqaoa_autotune": ([P, P, ctypes.c_int32, P, P, P, P, P], ctypes.c_int),
    "paraqaoa_schedule": ([ctypes.c_int32] * 9 + [P, P], ctypes.c_int),
    "paraqaoa_set_schedule": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32], ctypes.c_int),
    "paraqaoa_profile_enable": ([P, ctypes.c_int32], ctypes.c_int),
    "paraqaoa_profile_classes": ([P, ctypes.c_uint32], ctypes.c_int),
    "paraqaoa_profile_read": ([P, ctypes.c_int32, P, P, P], ctypes.c_int),
    "paraqaoa_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "paraqaoa_topk_noalloc": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, P, P, P], ctypes.c_int),
    "paraqaoa_features": ([P, P, P, ctypes.c_int32, P], ctypes.c_int),
    "paraqaoa_simulate_tc": ([P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_uint32, ctypes.c_int32,
                              ctypes.c_int32], ctypes.c_int),
    "paraqaoa_solve_plain": ([P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P], ctypes.c_int),
    "paraqaoa_angle_search": ([P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_double, ctypes.c_double, P, P, P], ctypes.c_int),
    "paraqaoa_final_topk": ([P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_uint32,
                             P, P, P], ctypes.c_int),
    "paraqaoa_set_wait_limit": ([P, ctypes.c_int64], ctypes.c_int),
    "paraqaoa_set_persistent": ([P, ctypes.c_int32], ctypes.c_int),
    "paraqaoa_set_halved": ([P, ctypes.c_int32], ctypes.c_int),
    "paraqaoa_probe_peaks": ([ctypes.c_int, P, P], ctypes.c_int),
    "paraqaoa_probe_streams": ([ctypes.c_int, ctypes.c_int64, P, P, P], ctypes.c_int),
    "paraqaoa_set_merge_fill": ([P, ctypes.c_int32, P], ctypes.c_int),
    "paraqaoa_pei": ([ctypes.c_double] * 4 + [P, P], ctypes.c_int),
    "paraqaoa_mlp_param_count": ([ctypes.c_int32], ctypes.c_int64),
    "paraqaoa_mlp_create": ([P, ctypes.c_int32, P, ctypes.POINTER(P)], ctypes.c_int),
    "paraqaoa_mlp_free": ([P], None),
    "paraqaoa_mlp_get_params": ([P, P], ctypes.c_int),
    "paraqaoa_mlp_grad": ([P, P, P, ctypes.c_int32, P, P], ctypes.c_int),
    "paraqaoa_mlp_train": ([P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P, P],
                           ctypes.c_int),
    "paraqaoa_mlp_predict": ([P, P, ctypes.c_int32, P, P], ctypes.c_int),
    "paraqaoa_mlp_reference": ([P, P, P], ctypes.c_int),
    "paraqaoa_solve_learned": ([P, P, P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_double, P, P, P, P],
                               ctypes.c_int),
}


def declared_symbols() -> list[str]:
    """Every function the public header declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(paraqaoa_[a-z_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load the CUDA library (build it first with build.py). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: run `python -m paper_2603_26232_gb300.native_build` "
                          "(the CUDA library is required; there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc: int, what: str):
    if rc != OK:
        raise ParaQAOAError(rc, what)


def strerror(code: int) -> str:
    return load().paraqaoa_strerror(code).decode()


# --------------------------------------------------------------------- objects
class Graph:
    """Host CSR arrays kept alive for the C struct that points into them."""

    def __init__(self, n: int, row_ptr, col, w):
        self.n = int(n)
        self.row_ptr = _arr(row_ptr, np.int64)
        self.col = _arr(col, np.int32)
        self.w = _arr(w, np.int32)
        self.csr = Csr(self.n, int(self.row_ptr[-1]), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.w))

    @classmethod
    def of(cls, g):
        return g if isinstance(g, Graph) else cls(g.n, g.row_ptr, g.col, g.w)


def paraqaoa_create(device: int = 0, hbm_budget: int = 0):
    h = P()
    _check(load().paraqaoa_create(ctypes.byref(h), int(device), int(hbm_budget)), "paraqaoa_create")
    return h


def paraqaoa_destroy(ctx):
    load().paraqaoa_destroy(ctx)


def paraqaoa_set_stream(ctx, stream_handle: int | None):
    _check(load().paraqaoa_set_stream(ctx, stream_handle), "paraqaoa_set_stream")


def paraqaoa_partition(g: Graph, M: int, mode: int = PART_BALANCED, sizes=None):
    h = P()
    sz = None if sizes is None else _arr(sizes, np.int32)
    _check(load().paraqaoa_partition(ctypes.byref(g.csr), int(M), int(mode), _ptr(sz), ctypes.byref(h)),
           "paraqaoa_partition")
    return h


def paraqaoa_part_free(part):
    load().paraqaoa_part_free(part)


def paraqaoa_part_info(part):
    M = np.zeros(1, np.int32)
    _check(load().paraqaoa_part_info(part, _ptr(M), None, None, None, None), "paraqaoa_part_info")
    m = int(M[0])
    first = np.zeros(m, np.int32)
    size = np.zeros(m, np.int32)
    edges = np.zeros(m, np.int64)
    weight = np.zeros(m, np.int64)
    _check(load().paraqaoa_part_info(part, None, _ptr(first), _ptr(size), _ptr(edges), _ptr(weight)),
           "paraqaoa_part_info")
    return first, size, edges, weight


def paraqaoa_part_edges(part, pid: int, count: int):
    u = np.zeros(count, np.int32)
    v = np.zeros(count, np.int32)
    w = np.zeros(count, np.int32)
    _check(load().paraqaoa_part_edges(part, int(pid), _ptr(u), _ptr(v), _ptr(w)), "paraqaoa_part_edges")
    return u, v, w


def paraqaoa_shard_plan(part, world: int, p: int, evals=None):
    """Rank of each part (longest processing time first) and each rank's load."""
    M = int(paraqaoa_part_info(part)[0].size)
    ev = None if evals is None else _arr(evals, np.float64)
    if ev is not None and ev.size != M:
        raise ValueError("evals must hold one entry per part")
    rank = np.zeros(M, np.int32)
    loads = np.zeros(int(world), np.float64)
    _check(load().paraqaoa_shard_plan(part, int(world), int(p), _ptr(ev), _ptr(rank), _ptr(loads)),
           "paraqaoa_shard_plan")
    return rank, loads


def paraqaoa_part_upload(ctx, part, force: bool = False):
    _check(load().paraqaoa_part_upload(ctx, part, 1 if force else 0), "paraqaoa_part_upload")


def paraqaoa_cut_table(ctx, part, pid: int, n: int) -> np.ndarray:
    out = np.zeros(1 << n, np.uint16)
    _check(load().paraqaoa_cut_table(ctx, part, int(pid), _ptr(out)), "paraqaoa_cut_table")
    return out


def paraqaoa_simulate_batch(ctx, part, ids, p: int, gamma, beta, flags: int = SIM_EXPECT):
    ids = _arr(ids, np.int32)
    g = _arr(gamma, np.float64).reshape(len(ids), p)
    b = _arr(beta, np.float64).reshape(len(ids), p)
    _check(load().paraqaoa_simulate_batch(ctx, part, _ptr(ids), len(ids), int(p), _ptr(g), _ptr(b),
                                          int(flags)), "paraqaoa_simulate_batch")


def paraqaoa_expect(ctx, count: int) -> np.ndarray:
    out = np.zeros(count, np.float64)
    _check(load().paraqaoa_expect(ctx, int(count), _ptr(out)), "paraqaoa_expect")
    return out


def paraqaoa_topk(ctx, count: int, K: int, flags: int = TOPK_CANONICAL):
    z = np.zeros((count, K), np.uint32)
    pr = np.zeros((count, K), np.float32)
    _check(load().paraqaoa_topk(ctx, int(count), int(K), _ptr(z), _ptr(pr), int(flags)), "paraqaoa_topk")
    return z, pr


def paraqaoa_state(ctx, i: int, n: int) -> np.ndarray:
    out = np.zeros(2 << n, np.float32)
    _check(load().paraqaoa_state(ctx, int(i), _ptr(out)), "paraqaoa_state")
    return out.view(np.complex64)


def paraqaoa_merge(ctx, g: Graph, part, cand, K: int, L: int = 1, beam: int = 0):
    cand = _arr(cand, np.uint32)
    side = np.zeros(g.n, np.uint8)
    cut = np.zeros(1, np.int64)
    _check(load().paraqaoa_merge(ctx, ctypes.byref(g.csr), part, _ptr(cand), int(K), int(L), int(beam),
                                 _ptr(side), _ptr(cut)), "paraqaoa_merge")
    return side, int(cut[0])


def paraqaoa_grid_search(ctx, part, ids, points: int = 16, want_values: bool = False):
    ids = _arr(ids, np.int32)
    n = len(ids)
    g = np.zeros(n, np.float64)
    b = np.zeros(n, np.float64)
    best = np.zeros(n, np.float64)
    vals = np.zeros(n * points * points, np.float64) if want_values else None
    _check(load().paraqaoa_grid_search(ctx, part, _ptr(ids), n, int(points), _ptr(g), _ptr(b), _ptr(best),
                                       _ptr(vals)), "paraqaoa_grid_search")
    return g, b, best, (vals.reshape(n, points * points) if want_values else None)


def paraqaoa_optimize(ctx, part, ids, p: int, gamma0, beta0, steps: int = 32, lr: float = 0.02,
                      h: float = 1e-3):
    ids = _arr(ids, np.int32)
    n = len(ids)
    g = np.array(gamma0, dtype=np.float64).reshape(n, p).copy()
    b = np.array(beta0, dtype=np.float64).reshape(n, p).copy()
    val = np.zeros(n, np.float64)
    _check(load().paraqaoa_optimize(ctx, part, _ptr(ids), n, int(p), int(steps), float(lr), float(h),
                                    _ptr(g), _ptr(b), _ptr(val)), "paraqaoa_optimize")
    return g, b, val


def paraqaoa_autotune(ctx, part, p: int = 2):
    """Time the layer-pass schedule candidates per qubit count; returns
    {n: (tile_bits, register_bits, min_contiguous_qubits, split, tiles_per_cta_log2)} for n >= 15."""
    tb = np.zeros(31, np.int32)
    rb = np.zeros(31, np.int32)
    cm = np.zeros(31, np.int32)
    sp = np.zeros(31, np.int32)
    tp = np.zeros(31, np.int32)
    _check(load().paraqaoa_autotune(ctx, part, int(p), _ptr(tb), _ptr(rb), _ptr(cm), _ptr(sp), _ptr(tp)),
           "paraqaoa_autotune")
    return {n: (int(tb[n]), int(rb[n]), int(cm[n]), int(sp[n]), int(tp[n])) for n in range(15, 31)}


def paraqaoa_profile_enable(ctx, enable: bool = True):
    _check(load().paraqaoa_profile_enable(ctx, 1 if enable else 0), "paraqaoa_profile_enable")


def paraqaoa_profile_classes(ctx, mask: int):
    """Bracket only the kernel classes whose bit is set (bit k = KCLASS k)."""
    _check(load().paraqaoa_profile_classes(ctx, int(mask) & 0xFFFFFFFF), "paraqaoa_profile_classes")


def paraqaoa_profile_read(ctx, which: int):
    n = np.zeros(1, np.int64)
    ms = np.zeros(1, np.float64)
    by = np.zeros(1, np.float64)
    _check(load().paraqaoa_profile_read(ctx, int(which), _ptr(n), _ptr(ms), _ptr(by)), "paraqaoa_profile_read")
    return int(n[0]), float(ms[0]), float(by[0])


def paraqaoa_topk_noalloc(state_dev_ptr: int, n: int, K: int, out_z_dev_ptr: int, out_p_dev_ptr: int,
                          flags: int = TOPK_CANONICAL, stream_handle: int | None = None):
    """Top-K of one device-resident state with no device allocation; pointers
    are raw device addresses (e.g. tensor.data_ptr()). Enqueues only."""
    _check(load().paraqaoa_topk_noalloc(state_dev_ptr, int(n), int(K), int(flags), out_z_dev_ptr,
                                        out_p_dev_ptr, stream_handle), "paraqaoa_topk_noalloc")


# ---------------------------------------------------------------- learned angles
FEATURES = 64


def paraqaoa_features(ctx, part, ids) -> np.ndarray:
    ids = _arr(ids, np.int32)
    out = np.zeros((ids.size, FEATURES), np.float32)
    _check(load().paraqaoa_features(ctx, part, _ptr(ids), ids.size, _ptr(out)), "paraqaoa_features")
    return out


def paraqaoa_solve_plain(ctx, part, ids, p: int, steps: int = 32):
    ids = _arr(ids, np.int32)
    g = np.zeros((ids.size, p))
    b = np.zeros((ids.size, p))
    v = np.zeros(ids.size)
    _check(load().paraqaoa_solve_plain(ctx, part, _ptr(ids), ids.size, p, steps, _ptr(g), _ptr(b), _ptr(v)),
           "paraqaoa_solve_plain")
    return g, b, v


def paraqaoa_angle_search(ctx, part, ids, p: int, points: int = 16, steps: int = 32, lr: float = 0.02,
                          h: float = 1e-3):
    ids = _arr(ids, np.int32)
    g = np.zeros((ids.size, p))
    b = np.zeros((ids.size, p))
    v = np.zeros(ids.size)
    _check(load().paraqaoa_angle_search(ctx, part, _ptr(ids), ids.size, int(p), int(points), int(steps), float(lr),
                                        float(h), _ptr(g), _ptr(b), _ptr(v)), "paraqaoa_angle_search")
    return g, b, v


def paraqaoa_final_topk(ctx, part, ids, p: int, gamma, beta, K: int, flags: int = TOPK_CANONICAL):
    """Returns (<C>, z, probabilities) of the final states, z / P of shape count x K."""
    ids = _arr(ids, np.int32)
    g = _arr(gamma, np.float64)
    b = _arr(beta, np.float64)
    if g.size != ids.size * p or b.size != ids.size * p:
        raise ValueError("gamma/beta must hold count x p angles")
    ex = np.zeros(ids.size)
    z = np.zeros((ids.size, K), np.uint32)
    pr = np.zeros((ids.size, K), np.float32)
    _check(load().paraqaoa_final_topk(ctx, part, _ptr(ids), ids.size, int(p), _ptr(g), _ptr(b), int(K), int(flags),
                                      _ptr(ex), _ptr(z), _ptr(pr)), "paraqaoa_final_topk")
    return ex, z, pr


def paraqaoa_set_halved(ctx, enable: bool = True):
    _check(load().paraqaoa_set_halved(ctx, 1 if enable else 0), "paraqaoa_set_halved")


def paraqaoa_set_persistent(ctx, enable: bool = True):
    _check(load().paraqaoa_set_persistent(ctx, 1 if enable else 0), "paraqaoa_set_persistent")


def paraqaoa_pei(ar: float, t_alg: float, t_base: float, alpha: float = 1e-3):
    """(EF, PEI) of a run (Sec. 3.5)."""
    ef = ctypes.c_double(0.0)
    pei = ctypes.c_double(0.0)
    _check(load().paraqaoa_pei(float(ar), float(t_alg), float(t_base), float(alpha), ctypes.byref(ef),
                               ctypes.byref(pei)), "paraqaoa_pei")
    return ef.value, pei.value


def paraqaoa_set_merge_fill(ctx, enable: int = -1) -> int:
    """Set the exhaustive merge's fill mode (1 on, 0 off, -1 keep); returns the
    starting level the context's last exhaustive merge used."""
    lv = ctypes.c_int32(0)
    _check(load().paraqaoa_set_merge_fill(ctx, int(enable), ctypes.byref(lv)), "paraqaoa_set_merge_fill")
    return int(lv.value)


def paraqaoa_probe_peaks(device: int = 0):
    """(FP32 TFLOP/s, shared-memory TB/s) measured on the device."""
    f = ctypes.c_double(0.0)
    m = ctypes.c_double(0.0)
    _check(load().paraqaoa_probe_peaks(int(device), ctypes.byref(f), ctypes.byref(m)), "paraqaoa_probe_peaks")
    return f.value, m.value


def paraqaoa_probe_streams(device: int = 0, nbytes: int = 1 << 31):
    """(write-only, read-only, copy) HBM GB/s measured on the device over
    buffers of nbytes each."""
    w, r, c = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().paraqaoa_probe_streams(int(device), int(nbytes), ctypes.byref(w), ctypes.byref(r), ctypes.byref(c)),
           "paraqaoa_probe_streams")
    return w.value, r.value, c.value


def paraqaoa_set_wait_limit(ctx, ns: int):
    _check(load().paraqaoa_set_wait_limit(ctx, int(ns)), "paraqaoa_set_wait_limit")


def paraqaoa_mlp_param_count(p: int) -> int:
    return int(load().paraqaoa_mlp_param_count(p))


def paraqaoa_mlp_create(ctx, p: int, init_params):
    w = _arr(init_params, np.float32)
    if w.size != paraqaoa_mlp_param_count(p):
        raise ValueError("init_params has the wrong size")
    out = P()
    _check(load().paraqaoa_mlp_create(ctx, p, _ptr(w), ctypes.byref(out)), "paraqaoa_mlp_create")
    return out


def paraqaoa_mlp_free(mlp):
    load().paraqaoa_mlp_free(mlp)


def paraqaoa_mlp_get_params(mlp, p: int) -> np.ndarray:
    out = np.zeros(paraqaoa_mlp_param_count(p), np.float32)
    _check(load().paraqaoa_mlp_get_params(mlp, _ptr(out)), "paraqaoa_mlp_get_params")
    return out


def paraqaoa_mlp_grad(mlp, p: int, X, T):
    X = _arr(X, np.float32)
    T = _arr(T, np.float32)
    g = np.zeros(paraqaoa_mlp_param_count(p), np.float32)
    loss = ctypes.c_double(0.0)
    _check(load().paraqaoa_mlp_grad(mlp, _ptr(X), _ptr(T), X.shape[0], _ptr(g), ctypes.byref(loss)),
           "paraqaoa_mlp_grad")
    return g, loss.value


def paraqaoa_mlp_train(mlp, X, T, epochs: int, batch: int, lr: float, order):
    X = _arr(X, np.float32)
    T = _arr(T, np.float32)
    order = _arr(order, np.int32)
    losses = np.zeros(epochs)
    _check(load().paraqaoa_mlp_train(mlp, _ptr(X), _ptr(T), X.shape[0], epochs, batch, lr, _ptr(order),
                                     _ptr(losses)), "paraqaoa_mlp_train")
    return losses


def paraqaoa_mlp_predict(mlp, p: int, X):
    X = _arr(X, np.float32)
    g = np.zeros((X.shape[0], p))
    b = np.zeros((X.shape[0], p))
    _check(load().paraqaoa_mlp_predict(mlp, _ptr(X), X.shape[0], _ptr(g), _ptr(b)), "paraqaoa_mlp_predict")
    return g, b


def paraqaoa_mlp_reference(mlp, p: int):
    g = np.zeros(p)
    b = np.zeros(p)
    _check(load().paraqaoa_mlp_reference(mlp, _ptr(g), _ptr(b)), "paraqaoa_mlp_reference")
    return g, b


def paraqaoa_solve_learned(ctx, part, ids, mlp, p: int, fallback_steps: int = 32, tol: float = 0.0):
    """Returns angles, <C> and per-part verdicts (0 network, 1 plain fallback, 2 reference)."""
    ids = _arr(ids, np.int32)
    g = np.zeros((ids.size, p))
    b = np.zeros((ids.size, p))
    v = np.zeros(ids.size)
    fb = np.zeros(ids.size, np.int32)
    _check(load().paraqaoa_solve_learned(ctx, part, _ptr(ids), ids.size, mlp, fallback_steps, float(tol), _ptr(g),
                                         _ptr(b), _ptr(v), _ptr(fb)), "paraqaoa_solve_learned")
    return g, b, v, fb


def paraqaoa_simulate_tc(ctx, part, ids, p: int, gamma, beta, flags: int = SIM_EXPECT, precision: int = TC_FP16,
                         block_qubits: int = 7):
    ids = _arr(ids, np.int32)
    g = _arr(gamma, np.float64)
    b = _arr(beta, np.float64)
    if g.size != ids.size * p or b.size != ids.size * p:
        raise ValueError("gamma/beta must hold count x p angles")
    _check(load().paraqaoa_simulate_tc(ctx, part, _ptr(ids), ids.size, int(p), _ptr(g), _ptr(b), int(flags),
                                       int(precision), int(block_qubits)), "paraqaoa_simulate_tc")


PASS_FIELDS = ("c", "s", "mix_lo", "layerA", "layerP", "layerB", "init", "store", "expect", "last", "split")


def paraqaoa_schedule(n: int, p: int, tile_bits: int, reg_bits: int, c_min: int = 3, split: int = 0,
                      keep: bool = False, expect: bool = True):
    """The layer-pass schedule (no context, no GPU): a list of dicts with PASS_FIELDS."""
    cnt = np.zeros(1, np.int32)
    _check(load().paraqaoa_schedule(int(n), int(p), int(tile_bits), int(reg_bits), int(c_min), int(split),
                                    int(bool(keep)), int(bool(expect)), 0, None, _ptr(cnt)), "paraqaoa_schedule")
    out = np.zeros((max(int(cnt[0]), 1), len(PASS_FIELDS)), np.int32)
    _check(load().paraqaoa_schedule(int(n), int(p), int(tile_bits), int(reg_bits), int(c_min), int(split),
                                    int(bool(keep)), int(bool(expect)), int(cnt[0]), _ptr(out), _ptr(cnt)),
           "paraqaoa_schedule")
    return [dict(zip(PASS_FIELDS, (int(v) for v in row))) for row in out[:int(cnt[0])]]


def paraqaoa_set_schedule(ctx, n: int, tile_bits: int, reg_bits: int, c_min: int = 3, split: int = 0,
                          tiles_per_cta_log2: int = 0):
    _check(load().paraqaoa_set_schedule(ctx, int(n), int(tile_bits), int(reg_bits), int(c_min), int(split),
                                        int(tiles_per_cta_log2)), "paraqaoa_set_schedule")
