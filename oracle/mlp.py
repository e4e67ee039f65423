"""Learned QAOA angles: subgraph features and the angle MLP -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy reference for the learned-angle part of the CUDA path. Only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use it.

The paper leaves the choice of initial angles open and notes that it matters
(Sec. 2.2: deeper circuits improve the approximation ratio, and the
optimiser's starting point affects how well it does). The learned part
predicts, from cheap features of a subgraph, the depth-p angles that the
plain optimiser (grid search, then fixed-iteration Adam; INTERP between
depths) finds for it, so most subgraphs skip that optimiser.

Precision model (the one the CUDA kernels implement): FP32 master weights;
every matrix product takes BF16 operands (round to nearest even) and
accumulates in FP32; biases, ReLU masks, the loss and Adam are FP32. With
``bf16=True`` the oracle rounds the same operands at the same points and
does everything else in FP64, so the two sides differ only by FP32 versus
FP64 accumulation and by rare one-ulp BF16 rounding differences.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss,
torch.autograd and torch.optim.Adam in float64, torch's bfloat16 rounding,
and networkx for the graph statistics behind the features.
"""
from __future__ import annotations

import numpy as np

F = 64          # feature count
HID = 256       # hidden width


# ------------------------------------------------------------------ features
def features(n: int, eu, ev, ew) -> np.ndarray:
    """64 features of one subgraph with n vertices and edge list (eu, ev, ew).

    Isolated vertices are left out first: a vertex without edges contributes
    nothing to C(z), its qubit's mixer commutes with everything else and the
    phase, and so neither <C> nor the best angles depend on it. With m the
    number of vertices that have at least one edge (all features 0 when m = 0):

      [0] m / 32                 [1] |E| / C(m,2)            [2] mean w / 16
      [3] std w / 16 (population) [4] mean degree / m        [5] std degree / m
      [6] max degree / m         [7] min degree / m
      [8..24)  degree histogram, bin min(deg, 15), counts / m
      [24..40) weight histogram, bin min(w, 16) - 1, counts / |E|
      [40..56) weighted-degree histogram, bin min(15, floor(16 D_u / (max_v D_v + 1))), counts / m
      [56] triangles / C(m,3)    [57] total weight / (10 C(m,2))    [58..64) 0

    Degrees and weighted degrees D run over the m non-isolated vertices.
    C(k, j) is the binomial coefficient (0 when k < j, and then the feature is 0).
    """
    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    ew = np.asarray(ew, np.int64)
    f = np.zeros(F, np.float64)
    E = eu.size
    deg = np.zeros(n, np.int64)
    wdeg = np.zeros(n, np.int64)
    adj = [set() for _ in range(n)]
    for a, b, w in zip(eu, ev, ew):
        deg[a] += 1
        deg[b] += 1
        wdeg[a] += w
        wdeg[b] += w
        adj[a].add(int(b))
        adj[b].add(int(a))
    keep = deg > 0
    m = int(keep.sum())
    if m == 0:
        return f
    deg, wdeg = deg[keep], wdeg[keep]
    pairs = m * (m - 1) / 2.0
    triples = m * (m - 1) * (m - 2) / 6.0
    f[0] = m / 32.0
    f[1] = E / pairs
    mw = ew.mean()
    f[2] = mw / 16.0
    f[3] = np.sqrt(max((ew.astype(np.float64) ** 2).mean() - mw * mw, 0.0)) / 16.0
    md = deg.mean()
    f[4] = md / m
    f[5] = np.sqrt(max((deg.astype(np.float64) ** 2).mean() - md * md, 0.0)) / m
    f[6] = deg.max() / m
    f[7] = deg.min() / m
    for d in deg:
        f[8 + min(int(d), 15)] += 1.0
    f[8:24] /= m
    for w in ew:
        f[24 + min(int(w), 16) - 1] += 1.0
    f[24:40] /= E
    dmax = int(wdeg.max())
    for d in wdeg:
        f[40 + min(15, (16 * int(d)) // (dmax + 1))] += 1.0
    f[40:56] /= m
    tri = 0
    for a, b in zip(eu, ev):
        tri += len(adj[int(a)] & adj[int(b)])
    tri //= 3
    f[56] = tri / triples if triples > 0 else 0.0
    f[57] = ew.sum() / (10.0 * pairs)
    return f


# ------------------------------------------------------------------ BF16
def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    returned as FP64. One rounding from the FP64 input."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)                      # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


# ------------------------------------------------------------------ network
def param_shapes(p: int):
    """(name, shape) of the parameters in storage order: W1[64x256], b1[256],
    W2[256x256], b2[256], W3[256x2p], b3[2p]; W is (in x out), row-major."""
    return [("W1", (F, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
            ("W3", (HID, 2 * p)), ("b3", (2 * p,))]


def param_count(p: int) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(p))


def unpack(flat, p: int) -> dict:
    out, o = {}, 0
    flat = np.asarray(flat, np.float64)
    for name, shp in param_shapes(p):
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(d: dict, p: int) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in param_shapes(p)])


def forward(params: dict, X, bf: bool = True):
    """Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3, rows of X are samples.
    With bf=True the operands of each product are rounded to BF16 first."""
    r = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    X = np.asarray(X, np.float64)
    Xb = r(X)
    Z1 = Xb @ r(params["W1"]) + params["b1"]
    H1 = np.maximum(Z1, 0.0)
    H1b = r(H1)
    Z2 = H1b @ r(params["W2"]) + params["b2"]
    H2 = np.maximum(Z2, 0.0)
    H2b = r(H2)
    Y = H2b @ r(params["W3"]) + params["b3"]
    cache = dict(Xb=Xb, Z1=Z1, H1b=H1b, Z2=Z2, H2b=H2b)
    return Y, cache


def loss_and_grad(params: dict, X, T, bf: bool = True):
    """Mean squared error over all rows x outputs, L = sum (Y - T)^2 / (rows * 2p),
    and its gradient by the chain rule through forward(). The backward
    products also take BF16 operands when bf=True."""
    r = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    T = np.asarray(T, np.float64)
    Y, c = forward(params, X, bf)
    N = Y.size
    D = Y - T
    L = float((D * D).sum() / N)
    dY = 2.0 * D / N
    dYb = r(dY)
    g = {}
    g["W3"] = c["H2b"].T @ dYb
    g["b3"] = dY.sum(axis=0)
    dH2 = dYb @ r(params["W3"]).T
    dZ2 = dH2 * (c["Z2"] > 0)
    dZ2b = r(dZ2)
    g["W2"] = c["H1b"].T @ dZ2b
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2b @ r(params["W2"]).T
    dZ1 = dH1 * (c["Z1"] > 0)
    dZ1b = r(dZ1)
    g["W1"] = c["Xb"].T @ dZ1b
    g["b1"] = dZ1.sum(axis=0)
    return L, g


class Adam:
    """Adam (Kingma and Ba, 2015) with bias correction, one state per parameter."""

    def __init__(self, flat_size: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(flat_size)
        self.v = np.zeros(flat_size)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, w: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - self.lr * mh / (np.sqrt(vh) + self.eps)


def train(flat0, p: int, X, T, order, batch: int, lr: float, bf: bool = True):
    """Minibatch Adam: epoch e visits rows order[e] in consecutive slices of
    `batch` (the last slice may be shorter). Returns the final flat
    parameters and the mean minibatch loss of each epoch."""
    w = np.asarray(flat0, np.float64).copy()
    opt = Adam(w.size, lr)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    losses = []
    for perm in order:
        ls = []
        for s in range(0, len(perm), batch):
            idx = perm[s:s + batch]
            L, g = loss_and_grad(unpack(w, p), X[idx], T[idx], bf)
            w = opt.step(w, pack(g, p))
            ls.append(L)
        losses.append(float(np.mean(ls)))
    return w, np.asarray(losses)


def predict(flat, p: int, X, bf: bool = True):
    """Angles (gamma[rows x p], beta[rows x p]) from the network output [gamma | beta]."""
    Y, _ = forward(unpack(flat, p), X, bf)
    return Y[:, :p], Y[:, p:]
