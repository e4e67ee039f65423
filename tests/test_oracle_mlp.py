"""Pins of the learned-angle oracle (oracle/mlp.py) to things other than itself:
finite differences, torch.autograd / torch.optim.Adam in float64, torch's
bfloat16 rounding, and networkx graph statistics."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

torch = pytest.importorskip("torch")


def _net(p=2, seed=3, rows=24):
    flat = synth.mlp_init(p, seed).astype(np.float64)
    # non-zero biases so that every bias gradient path is exercised
    rng = np.random.default_rng(seed)
    d = mlp.unpack(flat, p)
    for k in ("b1", "b2", "b3"):
        d[k] = rng.normal(0, 0.05, d[k].shape)
    X = rng.uniform(0, 1, (rows, mlp.F))
    T = rng.normal(0, 1, (rows, 2 * p))
    return d, X, T


def test_gradient_matches_central_differences():
    p = 2
    d, X, T = _net(p)
    L, g = mlp.loss_and_grad(d, X, T, bf=False)
    rng = np.random.default_rng(0)
    h = 1e-6
    for name, shp in mlp.param_shapes(p):
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shp)
            dp = {k: v.copy() for k, v in d.items()}
            dm = {k: v.copy() for k, v in d.items()}
            dp[name][idx] += h
            dm[name][idx] -= h
            fd = (mlp.loss_and_grad(dp, X, T, bf=False)[0] - mlp.loss_and_grad(dm, X, T, bf=False)[0]) / (2 * h)
            an = g[name][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (name, idx, fd, an)


def test_gradient_matches_torch_autograd():
    p = 3
    d, X, T = _net(p, seed=5, rows=40)
    L, g = mlp.loss_and_grad(d, X, T, bf=False)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in d.items()}
    x = torch.tensor(X, dtype=torch.float64)
    y = torch.relu(torch.relu(x @ tp["W1"] + tp["b1"]) @ tp["W2"] + tp["b2"]) @ tp["W3"] + tp["b3"]
    lt = torch.nn.functional.mse_loss(y, torch.tensor(T, dtype=torch.float64))
    lt.backward()
    assert abs(lt.item() - L) <= 1e-12 * max(1.0, L)
    for k in d:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-14)


def test_adam_matches_torch():
    p = 1
    d, X, T = _net(p, seed=7)
    w = mlp.pack(d, p)
    opt = mlp.Adam(w.size, lr=1e-3)
    tw = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    topt = torch.optim.Adam([tw], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(3):
        _, g = mlp.loss_and_grad(mlp.unpack(w, p), X, T, bf=False)
        gf = mlp.pack(g, p)
        w = opt.step(w, gf)
        topt.zero_grad()
        tw.grad = torch.tensor(gf, dtype=torch.float64)
        topt.step()
    np.testing.assert_allclose(w, tw.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 5000), rng.uniform(-300, 300, 5000)])
    x32 = x.astype(np.float32)  # float32 inputs: torch rounds float32 -> bfloat16 once, as the GPU does
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32.astype(np.float64)), ref)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_bf16_forward_close_to_fp64_forward():
    # BF16 operands keep 8 significant bits: outputs agree to a few 2^-8 relative
    d, X, T = _net(2, seed=9, rows=32)
    y64, _ = mlp.forward(d, X, bf=False)
    y16, _ = mlp.forward(d, X, bf=True)
    assert np.max(np.abs(y16 - y64)) <= 4 * 2.0 ** -8 * np.max(np.abs(y64)) + 1e-6


def test_features_against_networkx():
    nx = pytest.importorskip("networkx")
    for seed, (n, pe, wmax) in enumerate([(12, 0.3, 10), (9, 0.8, 3), (15, 0.1, 1), (20, 0.05, 1)]):
        g = synth.erdos_renyi(n, pe, seed, wmax=wmax)
        f = mlp.features(n, g.eu, g.ev, g.ew)
        G = nx.Graph()
        for a, b, w in zip(g.eu, g.ev, g.ew):
            G.add_edge(int(a), int(b), weight=int(w))   # only vertices with edges
        m = G.number_of_nodes()
        assert m > 0
        deg = np.array([d for _, d in G.degree()])
        wdeg = np.array([d for _, d in G.degree(weight="weight")])
        ws = np.array([w for _, _, w in G.edges(data="weight")])
        assert f[0] == m / 32
        assert np.isclose(f[1], nx.density(G))
        assert np.isclose(f[2], ws.mean() / 16) and np.isclose(f[3], ws.std() / 16)
        assert np.isclose(f[4], deg.mean() / m) and np.isclose(f[5], deg.std() / m)
        assert f[6] == deg.max() / m and f[7] == deg.min() / m
        assert np.isclose(f[8:24].sum(), 1.0) and f[8] == 0.0
        for b in range(16):
            assert np.isclose(f[8 + b], np.sum(np.minimum(deg, 15) == b) / m)
            assert np.isclose(f[40 + b], np.sum(np.minimum(wdeg * 16 // (wdeg.max() + 1), 15) == b) / m)
        assert np.isclose(f[24:40].sum(), 1.0)
        tri = sum(nx.triangles(G).values()) // 3
        assert np.isclose(f[56], tri / (m * (m - 1) * (m - 2) / 6) if m > 2 else 0.0)
        assert np.isclose(f[57], ws.sum() / (10 * m * (m - 1) / 2))
        assert np.all(f[58:] == 0)


def test_features_closed_forms():
    # complete graph K_n with unit weights: every degree n-1, C(n,3) triangles
    n = 7
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    g = synth.from_edges(n, e)
    f = mlp.features(n, g.eu, g.ev, g.ew)
    assert f[1] == 1.0 and f[56] == 1.0 and f[8 + n - 1] == 1.0
    assert np.isclose(f[2], 1 / 16) and f[3] == 0.0 and f[24] == 1.0
    # a single edge: m = 2, density 1, both degrees 1
    f1 = mlp.features(5, [1], [3], [4])
    assert f1[0] == 2 / 32 and f1[1] == 1.0 and f1[9] == 1.0 and f1[24 + 3] == 1.0
    # edgeless graph: all zero
    assert np.count_nonzero(mlp.features(5, [], [], [])) == 0


def test_features_ignore_isolated_vertices():
    # isolated vertices change neither <C> nor the best angles, nor the features
    g = synth.erdos_renyi(10, 0.4, 3, wmax=10)
    f = mlp.features(10, g.eu, g.ev, g.ew)
    perm = np.array([0, 3, 5, 7, 11, 12, 14, 17, 20, 23])   # spread over 26 vertices
    f2 = mlp.features(26, perm[g.eu], perm[g.ev], g.ew)
    np.testing.assert_array_equal(f, f2)


def test_chain_of_graphs_parts_are_the_graphs():
    specs = synth.graph_specs(6, 5, 9, 0.2, 0.6, 11)
    G, sizes = synth.chain_of_graphs(specs, wmax=10)
    subs = oracle.subgraphs(G, len(sizes), 2, sizes)
    for (n, pe, s), sub in zip(specs, subs):
        g = synth.erdos_renyi(n, pe, s, wmax=10)
        assert sub.n == n
        np.testing.assert_array_equal(sub.eu, g.eu)
        np.testing.assert_array_equal(sub.ev, g.ev)
        np.testing.assert_array_equal(sub.ew, g.ew)


def test_training_reduces_loss_on_a_learnable_target():
    # targets that are an exact function of the inputs: the minibatch loss falls
    p = 1
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (128, mlp.F))
    T = np.stack([X[:, 0] + 0.5 * X[:, 1], X[:, 2] - X[:, 3]], axis=1)
    order = synth.epoch_orders(128, 6, 0)
    w, losses = mlp.train(synth.mlp_init(p, 0), p, X, T, order, 32, 3e-3, bf=False)
    assert losses[-1] < 0.2 * losses[0]
