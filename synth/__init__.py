"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no step of the method: it only draws graphs, size lists and
angles. Every random number comes from one counter-based generator, the
SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the m-th draw of stream ``key``
is ``mix(key + (m + 1) * 0x9E3779B97F4A7C15)``. Draw m is therefore a pure
function of (key, m), which lets numpy produce millions of draws at once and
gives the same numbers on any machine.

The evaluation graphs of the paper are Erdos-Renyi graphs (Section 4.1); the
NetworkX random stream it used is not reproduced here, so these graphs are
statistically equivalent, not identical.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream keys: each purpose draws from its own stream so that, e.g., changing
# the weight range does not change the edge set.
EDGE_STREAM = 0x45444745  # "EDGE"
WEIGHT_STREAM = 0x57474854  # "WGHT"
SIZES_STREAM = 0x53495a45  # "SIZE"
ANGLE_STREAM = 0x414e474c  # "ANGL"


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one stream: the first SplitMix64 output of (seed, stream)."""
    base = np.array([(int(seed) * 0x100000001B3 + int(stream)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(base + GOLDEN)[0]


def draws_u64(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of stream ``key`` as uint64."""
    m = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + m * GOLDEN)


def draws_unit(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of each draw."""
    return (draws_u64(key, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Graph:
    """Undirected weighted graph as a symmetric CSR (both directions stored).

    row_ptr int64[n+1], col int32[nnz], w int32[nnz]; no self-loops, w > 0,
    column indices sorted within each row.
    """

    def __init__(self, n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray):
        self.n = int(n)
        u = np.asarray(u, dtype=np.int64)
        v = np.asarray(v, dtype=np.int64)
        w = np.asarray(w, dtype=np.int64)
        assert np.all(u != v), "self-loop"
        a = np.concatenate([u, v])
        b = np.concatenate([v, u])
        ww = np.concatenate([w, w])
        order = np.lexsort((b, a))
        a, b, ww = a[order], b[order], ww[order]
        counts = np.bincount(a, minlength=self.n) if a.size else np.zeros(self.n, np.int64)
        self.row_ptr = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(counts, out=self.row_ptr[1:])
        self.col = b.astype(np.int32)
        self.w = ww.astype(np.int32)
        # canonical edge list u < v
        keep = u < v
        eu = np.where(keep, u, v)
        ev = np.where(keep, v, u)
        order = np.lexsort((ev, eu))
        self.eu = eu[order].astype(np.int32)
        self.ev = ev[order].astype(np.int32)
        self.ew = w[order].astype(np.int32)

    @property
    def num_edges(self) -> int:
        return int(self.eu.size)

    @property
    def total_weight(self) -> int:
        return int(self.ew.astype(np.int64).sum())


def erdos_renyi(n: int, p: float, seed: int, wmax: int = 1) -> Graph:
    """G(n, p): pair (i, j), i < j, in lexicographic order is pair number m;
    the edge exists when draw m of the edge stream is below p. Its weight is
    1 + (draw m of the weight stream mod wmax), i.e. uniform in {1..wmax}."""
    ke = stream_key(seed, EDGE_STREAM)
    kw = stream_key(seed, WEIGHT_STREAM)
    us, vs, ws = [], [], []
    m0 = 0
    for i in range(n - 1):
        cnt = n - 1 - i
        u = draws_unit(ke, m0, cnt)
        hit = np.nonzero(u < p)[0]
        if hit.size:
            j = i + 1 + hit
            us.append(np.full(hit.size, i, dtype=np.int64))
            vs.append(j.astype(np.int64))
            if wmax > 1:
                wd = draws_u64(kw, m0, cnt)[hit] % np.uint64(wmax)
                ws.append(1 + wd.astype(np.int64))
            else:
                ws.append(np.ones(hit.size, dtype=np.int64))
        m0 += cnt
    if us:
        return Graph(n, np.concatenate(us), np.concatenate(vs), np.concatenate(ws))
    return Graph(n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64))


def from_edges(n: int, edges, weights=None) -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(e), np.int64) if weights is None else np.asarray(weights, np.int64)
    return Graph(n, e[:, 0], e[:, 1], w)


def uneven_sizes(num_vertices: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Part sizes drawn uniformly from {lo..hi} until they cover num_vertices
    vertices with one shared vertex between neighbours (sum(sizes) - (M-1) =
    num_vertices); the last size is trimmed (and kept >= 2) to land exactly."""
    key = stream_key(seed, SIZES_STREAM)
    sizes = []
    covered = 1  # the first part's shared-vertex bookkeeping: parts add size-1 new vertices
    m = 0
    while covered < num_vertices:
        s = lo + int(draws_u64(key, m, 1)[0] % np.uint64(hi - lo + 1))
        m += 1
        new = s - 1
        if covered + new >= num_vertices:
            s = num_vertices - covered + 1
            if s < 2:
                s = 2
            sizes.append(s)
            covered = num_vertices
            break
        sizes.append(s)
        covered += new
    if not sizes:
        sizes = [num_vertices]
    return np.asarray(sizes, dtype=np.int32)


def random_angles(count: int, p: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """gamma in [0, pi), beta in [-pi/4, pi/4): count x p each (float64)."""
    key = stream_key(seed, ANGLE_STREAM)
    u = draws_unit(key, 0, 2 * count * p).reshape(2, count, p)
    return u[0] * np.pi, (u[1] - 0.5) * (np.pi / 2)



MLP_STREAM = 0x4d4c5049  # "MLPI"
ORDER_STREAM = 0x4f524452  # "ORDR"
GRAPHS_STREAM = 0x47525048  # "GRPH"


def mlp_init(p: int, seed: int, fan=((64, 256), (256, 256), (256, None))) -> np.ndarray:
    """Initial parameters of the 64 -> 256 -> 256 -> 2p angle network, flat in
    storage order (W1, b1, W2, b2, W3, b3; W as in x out, row-major): weights
    uniform in +-sqrt(6 / (in + out)) (Glorot and Bengio, 2010), biases 0.
    Values are rounded to float32 so every consumer starts from the same numbers."""
    key = stream_key(seed, MLP_STREAM)
    out, m = [], 0
    for fi, fo in fan:
        fo = 2 * p if fo is None else fo
        a = np.sqrt(6.0 / (fi + fo))
        u = draws_unit(key, m, fi * fo)
        m += fi * fo
        out.append(((2.0 * u - 1.0) * a).astype(np.float32))
        out.append(np.zeros(fo, np.float32))
    return np.concatenate(out).astype(np.float32)


def epoch_orders(rows: int, epochs: int, seed: int) -> np.ndarray:
    """One permutation of range(rows) per epoch (sort keys drawn per row)."""
    key = stream_key(seed, ORDER_STREAM)
    d = draws_u64(key, 0, rows * epochs).reshape(epochs, rows)
    return np.argsort(d, axis=1, kind="stable").astype(np.int32)


def graph_specs(count: int, n_lo: int, n_hi: int, p_lo: float, p_hi: float, seed: int):
    """Per random subgraph: (n, edge probability, graph seed), n uniform in
    {n_lo..n_hi}, probability uniform in [p_lo, p_hi); graph seeds are
    seed * 1_000_003 + index."""
    key = stream_key(seed, GRAPHS_STREAM)
    d = draws_u64(key, 0, 2 * count).reshape(2, count)
    ns = n_lo + (d[0] % np.uint64(n_hi - n_lo + 1)).astype(np.int64)
    ps = p_lo + (d[1] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * (p_hi - p_lo)
    return [(int(n), float(pe), int(seed) * 1_000_003 + i) for i, (n, pe) in enumerate(zip(ns, ps))]


def chain_of_graphs(specs, wmax: int = 10):
    """Place independent G(n, P) graphs on a chain of vertex ranges that
    overlap in one vertex, [o_i, o_i + n_i) with o_{i+1} = o_i + n_i - 1, so
    that the SIZES partition with sizes n_i recovers graph i as part i
    (no edge of graph i+1 has both ends in part i and vice versa).
    Returns (whole graph, sizes)."""
    us, vs, ws, sizes = [], [], [], []
    o = 0
    for n, pe, s in specs:
        g = erdos_renyi(n, pe, s, wmax=wmax)
        us.append(g.eu.astype(np.int64) + o)
        vs.append(g.ev.astype(np.int64) + o)
        ws.append(g.ew.astype(np.int64))
        sizes.append(n)
        o += n - 1
    total = o + 1
    return Graph(total, np.concatenate(us), np.concatenate(vs), np.concatenate(ws)), np.asarray(sizes, np.int32)
