"""Pins of the CPU oracle to facts that do not come from the oracle itself:
closed forms, dense matrix exponentials, library graph routines, symmetry
laws, brute force and the paper's worked examples."""
import itertools
import json
import os

import networkx as nx
import numpy as np
import pytest
import scipy.linalg as sla

import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def sub_of(g, orc):
    return orc.Subgraph(0, g.n, g.eu, g.ev, g.ew)


def nx_graph(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for a, b, w in zip(g.eu, g.ev, g.ew):
        G.add_edge(int(a), int(b), weight=int(w))
    return G


# ------------------------------------------------------------------ cut table
def test_cut_table_matches_networkx_cut_size(orc):
    g = synth.erdos_renyi(9, 0.45, 11, wmax=10)
    G = nx_graph(g)
    ct = orc.cut_table(sub_of(g, orc))
    for z in [0, 1, 5, 77, 200, 311, 511]:
        S = [v for v in range(g.n) if (z >> v) & 1]
        assert ct[z] == nx.cut_size(G, S, weight="weight")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cut_table_symmetry_and_zero(orc, seed):
    g = synth.erdos_renyi(10, 0.5, seed, wmax=7)
    ct = orc.cut_table(sub_of(g, orc))
    full = (1 << g.n) - 1
    z = np.arange(1 << g.n)
    assert ct[0] == 0
    assert np.array_equal(ct, ct[full ^ z])


def test_cut_table_max_closed_forms(orc):
    # complete graph K_n: floor(n/2) * ceil(n/2)
    for n in range(2, 10):
        g = synth.from_edges(n, list(itertools.combinations(range(n), 2)))
        assert orc.cut_table(sub_of(g, orc)).max() == (n // 2) * ((n + 1) // 2)
    # cycles: n if even, n-1 if odd
    for n in range(3, 11):
        g = synth.from_edges(n, [(i, (i + 1) % n) for i in range(n)])
        assert orc.cut_table(sub_of(g, orc)).max() == (n if n % 2 == 0 else n - 1)
    # bipartite (weighted): the whole weight
    g = synth.from_edges(7, [(0, 4), (0, 5), (1, 5), (2, 6), (3, 4), (3, 6)], [3, 1, 4, 1, 5, 9])
    assert orc.cut_table(sub_of(g, orc)).max() == 23
    # Petersen graph: maximum cut 12
    P = nx.petersen_graph()
    g = synth.from_edges(10, list(P.edges()))
    assert orc.cut_table(sub_of(g, orc)).max() == 12


def test_bruteforce_maxcut(orc):
    P = nx.petersen_graph()
    g = synth.from_edges(10, list(P.edges()))
    best, z = orc.bruteforce_maxcut(sub_of(g, orc))
    assert best == 12
    S = [v for v in range(10) if (z >> v) & 1]
    assert nx.cut_size(P, S) == 12
    assert (z >> 9) & 1 == 0


# ------------------------------------------------------------------ simulation
def _kron_all(ops):
    out = np.array([[1.0 + 0j]])
    for o in ops:
        out = np.kron(o, out)  # qubit 0 is the least significant factor
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_simulate_equals_dense_exponentials(orc, p):
    """|psi> = prod_l exp(-i b_l H_M) exp(-i g_l H_C) |+>^n with H_C the
    diagonal of networkx cut sizes and H_M = sum_j X_j built by Kronecker
    products; scipy expm supplies the exponentials."""
    g = synth.erdos_renyi(5, 0.6, 4, wmax=3)
    n = g.n
    G = nx_graph(g)
    diag = np.array([nx.cut_size(G, [v for v in range(n) if (z >> v) & 1], weight="weight")
                     for z in range(1 << n)], dtype=np.float64)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    I2 = np.eye(2, dtype=np.complex128)
    HM = sum(_kron_all([X if k == j else I2 for k in range(n)]) for j in range(n))
    gam, bet = synth.random_angles(1, p, 7 + p)
    psi = np.full(1 << n, 2 ** (-n / 2), dtype=np.complex128)
    for l in range(p):
        psi = np.exp(-1j * gam[0, l] * diag) * psi
        psi = sla.expm(-1j * bet[0, l] * HM) @ psi
    ours = orc.simulate(sub_of(g, orc), gam[0], bet[0])
    assert np.max(np.abs(ours - psi)) < 1e-12


def _closed_form_p1(g, gam, bet):
    """Wang, Hadfield, Jiang, Rieffel, PRA 97, 022304 (2018): p = 1 <C> of an
    unweighted graph, edge by edge (d = degree - 1, lam = common neighbours)."""
    adj = [set() for _ in range(g.n)]
    for a, b in zip(g.eu, g.ev):
        adj[a].add(b)
        adj[b].add(a)
    tot = 0.0
    for a, b in zip(g.eu, g.ev):
        du, dv, lam = len(adj[a]) - 1, len(adj[b]) - 1, len(adj[a] & adj[b])
        tot += (0.5 + 0.25 * np.sin(4 * bet) * np.sin(gam) * (np.cos(gam) ** du + np.cos(gam) ** dv)
                - 0.25 * np.sin(2 * bet) ** 2 * np.cos(gam) ** (du + dv - 2 * lam) * (1 - np.cos(2 * gam) ** lam))
    return tot


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_p1_closed_form(orc, seed):
    g = synth.erdos_renyi(11, 0.4, seed)
    s = sub_of(g, orc)
    gam, bet = synth.random_angles(3, 1, 100 + seed)
    for k in range(3):
        st = orc.simulate(s, gam[k], bet[k])
        assert abs(orc.expect_state(s, st) - _closed_form_p1(g, gam[k, 0], bet[k, 0])) < 1e-10


def test_single_edge(orc):
    g = synth.from_edges(2, [(0, 1)])
    s = sub_of(g, orc)
    for gam, bet in [(0.3, 0.2), (1.7, -0.6), (2.9, 0.77)]:
        st = orc.simulate(s, [gam], [bet])
        assert abs(orc.expect_state(s, st) - (0.5 + 0.5 * np.sin(4 * bet) * np.sin(gam))) < 1e-13


def test_zero_angles_give_half_weight(orc):
    g = synth.erdos_renyi(10, 0.5, 5, wmax=10)
    s = sub_of(g, orc)
    W = g.total_weight
    st = orc.simulate(s, [0.0, 0.0], [0.0, 0.0])
    assert abs(orc.expect_state(s, st) - W / 2) < 1e-9
    st = orc.simulate(s, [0.7, 1.3], [0.0, 0.0])  # beta = 0: phases only
    assert abs(orc.expect_state(s, st) - W / 2) < 1e-9


def test_norm_and_symmetries(orc):
    g = synth.erdos_renyi(10, 0.5, 6, wmax=10)
    s = sub_of(g, orc)
    gam, bet = synth.random_angles(1, 3, 9)
    st = orc.simulate(s, gam[0], bet[0])
    assert abs(np.vdot(st, st).real - 1) < 1e-12
    pr = np.abs(st) ** 2
    z = np.arange(1 << g.n)
    assert np.max(np.abs(pr - pr[((1 << g.n) - 1) ^ z])) < 1e-14  # P(z) = P(not z)
    st2 = orc.simulate(s, -gam[0], -bet[0])
    assert abs(orc.expect_state(s, st) - orc.expect_state(s, st2)) < 1e-10
    # beta period pi/2 and gamma period 2 pi (integer weights)
    st3 = orc.simulate(s, gam[0] + 2 * np.pi, bet[0] + np.pi / 2)
    assert abs(orc.expect_state(s, st) - orc.expect_state(s, st3)) < 1e-10


def test_edgeless_stays_uniform(orc):
    g = synth.from_edges(6, np.zeros((0, 2), int))
    s = sub_of(g, orc)
    st = orc.simulate(s, [0.4, 1.0], [0.3, -0.2])
    assert np.max(np.abs(np.abs(st) ** 2 - 1 / 64)) < 1e-14


def test_farhi_petersen_p1_optimum(orc):
    """Petersen graph: 3-regular with girth 5, so the p = 1 optimum per edge
    is 1/2 + 1/(3 sqrt 3) (Farhi et al. 2014)."""
    P = nx.petersen_graph()
    g = synth.from_edges(10, list(P.edges()))
    batch = orc.Batch([sub_of(g, orc)])
    gg, bb = np.meshgrid(np.linspace(0, np.pi, 181), np.linspace(-np.pi / 4, np.pi / 4, 91), indexing="ij")
    vals = orc.expect_batch(batch, np.zeros(gg.size, np.int32), gg.ravel(), bb.ravel())
    k = np.argmax(vals)
    g0, b0 = gg.ravel()[k], bb.ravel()[k]
    gf, bf, final = orc.adam_optimize(batch, [[g0]], [[b0]], orc.AdamConfig(steps=200, lr=0.002))
    per_edge = max(final[0], vals[k]) / 15
    assert abs(per_edge - GOLD["farhi_3regular_p1"]["per_edge"]) < 2e-5


# ------------------------------------------------------------------ top-K
@pytest.mark.parametrize("canonical", [True, False])
def test_topk_equals_full_sort(orc, canonical):
    g = synth.erdos_renyi(11, 0.5, 12, wmax=5)
    s = sub_of(g, orc)
    st = orc.simulate(s, [0.5, 0.9], [0.3, 0.1])
    K = 24
    z, pr = orc.topk(g.n, st, K, canonical)
    probs = np.abs(st) ** 2
    zz = np.arange(1 << g.n)
    if canonical:
        zz = zz[zz < (1 << (g.n - 1))]
    order = np.lexsort((zz, -probs[zz]))
    assert np.array_equal(z, zz[order[:K]])
    assert np.allclose(pr, probs[z], rtol=1e-14, atol=0)


# ------------------------------------------------------------------ partition
def test_partition_alg1_literal_worked_example(orc):
    ex = GOLD["alg1_literal"]
    first, size = orc.partition(ex["num_vertices"], ex["M"], mode=1)
    assert first.tolist() == ex["first"] and size.tolist() == ex["size"]


@pytest.mark.parametrize("nv,M,expect", [(20, 2, [11, 10]), (400, 21, [20] * 21), (16000, 640, [26] * 639 + [25])])
def test_partition_balanced_sizes(orc, nv, M, expect):
    first, size = orc.partition(nv, M, mode=0)
    assert size.tolist() == expect
    # Sec. 3.2 constraints: neighbours share exactly one vertex, all covered
    for i in range(M - 1):
        a = set(range(first[i], first[i] + size[i]))
        b = set(range(first[i + 1], first[i + 1] + size[i + 1]))
        assert len(a & b) == 1
    assert first[0] == 0 and first[-1] + size[-1] == nv
    assert max(size) <= int(np.ceil(nv / M)) + 1


def test_partition_sizes_mode(orc):
    sizes = synth.uneven_sizes(300, 12, 24, 1)
    first, size = orc.partition(300, len(sizes), mode=2, sizes=sizes)
    assert size.tolist() == sizes.tolist()
    assert first[-1] + size[-1] == 300
    with pytest.raises(ValueError):
        orc.partition(301, len(sizes), mode=2, sizes=sizes)


def test_get_subgraph_matches_networkx(orc):
    g = synth.erdos_renyi(60, 0.2, 3, wmax=10)
    G = nx_graph(g)
    subs = orc.subgraphs(g, 5)
    seen = set()
    for s in subs:
        H = G.subgraph(range(s.first, s.first + s.n))
        ref = sorted((min(a, b) - s.first, max(a, b) - s.first, d["weight"]) for a, b, d in H.edges(data=True))
        ours = sorted(zip(s.eu.tolist(), s.ev.tolist(), s.ew.tolist()))
        assert ours == ref
        seen |= {(s.first + a, s.first + b) for a, b, _ in ours}
    inter = orc.inter_edges(g, subs)
    assert len(seen) + len(inter) == g.num_edges
    assert not (seen & {(a, b) for a, b, _ in inter})


# ------------------------------------------------------------------ merge
def _bits(sv: str) -> int:
    return sum(1 << i for i, ch in enumerate(sv) if ch == "1")


def test_merge_paper_example(orc):
    ex = GOLD["dc_example"]
    g = synth.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
    first = [p[0] for p in ex["parts"]]
    size = [p[1] for p in ex["parts"]]
    want = np.array([int(c) for c in ex["merged"]], np.uint8)
    for second in (ex["candidates"][1], "".join("1" if c == "0" else "0" for c in ex["candidates"][1])):
        cand = np.array([[_bits(ex["candidates"][0])], [_bits(second)]], np.uint32)
        side, cut, leaves = orc.merge_exhaustive(g, first, size, cand, K=1, L=1)
        assert np.array_equal(side, want) or np.array_equal(side, 1 - want)
        assert cut == orc.cutval(g, side)


def _brute_merge(g, first, size, cand, K):
    best, arg = -1, None
    for tup in itertools.product(range(K), repeat=len(first)):
        side = np.zeros(g.n, np.uint8)
        for lvl, j in enumerate(tup):
            b = int(cand[lvl][j])
            f, s = first[lvl], size[lvl]
            if lvl > 0 and (b & 1) != side[f]:
                b = (~b) & ((1 << s) - 1)
            for v in range(s):
                side[f + v] = (b >> v) & 1
        S = [v for v in range(g.n) if side[v]]
        c = nx.cut_size(nx_graph(g), S, weight="weight")
        if c > best:
            best, arg = c, side.copy()
    return best, arg


@pytest.mark.parametrize("seed", [0, 1])
def test_merge_exhaustive_equals_brute_force(orc, seed):
    g = synth.erdos_renyi(16, 0.35, seed, wmax=4)
    first, size = orc.partition(g.n, 4)
    K = 3
    rng = np.random.default_rng(seed)
    cand = np.array([rng.integers(0, 1 << int(s), K) for s in size], dtype=np.uint32)
    best, arg = _brute_merge(g, first, size, cand, K)
    for L in (1, 2, 3):
        side, cut, leaves = orc.merge_exhaustive(g, first, size, cand, K, L)
        assert cut == best
        assert leaves == K ** len(first)
        ref = arg if arg[0] == 0 else 1 - arg
        assert np.array_equal(side, ref)
    # beam wide enough to keep every partial path equals the exhaustive merge
    side_b, cut_b = orc.merge_beam(g, first, size, cand, K, beam=K ** (len(first) - 1))
    assert cut_b == best and np.array_equal(side_b, side)
    # narrow beams never beat it and always report their own assignment's cut
    for B in (1, 2, 5):
        sb, cb = orc.merge_beam(g, first, size, cand, K, beam=B)
        assert cb <= best and cb == orc.cutval(g, sb)


# A hand-worked beam case (the beam reading of Sec. 3.4 for K^M beyond reach:
# keep the best B partial paths per level by the cut of the edges with both
# ends assigned, ties to the lexicographically smaller candidate tuple). Path
# 0-1 | 2-3 | 4-5 (unit weights) plus a weight-5 edge (1, 3) between levels 0
# and 1; parts {0,1,2}, {2,3,4}, {4,5,6}; K = 2 candidates per part with ties
# planted at levels 0 and 2, worked out by hand:
#   level 0: cand 0 = 0b010 (v1 in S), cand 1 = 0b001 (v0 in S): both cut
#            (0, 1), partial score 1 each -> a tie.
#   level 1: cand 0 = 0b111 has v2 = 1 against side[2] = 0, so it is taken
#            complemented (0b000); cand 1 = 0b010 (v3 in S).
#            (0,0): 1 + 0 + 5 (edge (1,3), v1 = 1, v3 = 0) = 6
#            (0,1): 1 + 1 (edge (2,3)) + 0 = 2
#            (1,0): 1 + 0 + 0 = 1;  (1,1): 1 + 1 + 5 = 7
#   level 2: cand 0 = 0b010 (v5 in S), cand 1 = 0b110 (v5, v6 in S): both cut
#            only (4, 5) -> +1 each, another tie (v6 has no edges).
# B = 1 keeps (0) at level 0 (the tie goes to the smaller tuple), then (0,0)
# with 6, then (0,0,0) with 7: side 0100010, cut 7. Picking the larger tuple
# on the level-0 tie would reach (1,1) and cut 8 instead; on the level-2 tie
# it would put v6 in S.
# B = 2 keeps both level-0 paths, then (1,1) = 7 and (0,0) = 6, then
# (1,1,0) = (1,1,1) = 8 > 7: (1,1,0), side 1001010, normalised so that
# vertex 0 is on side 0: 0110101, cut 8.
# (The case is stored in tests/golden/beam_hand_case.json for the GPU test.)
BEAM_HAND = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "beam_hand_case.json")))


def test_merge_beam_hand_worked_ties(orc):
    h = BEAM_HAND
    assert h["candidates"] == [[0b010, 0b001], [0b111, 0b010], [0b010, 0b110]]
    g = synth.from_edges(h["num_vertices"], h["edges"], h["weights"])
    first, size = orc.partition(h["num_vertices"], h["M"])
    assert list(first) == [0, 2, 4] and list(size) == [3, 3, 3]
    cand = np.array(h["candidates"], np.uint32)
    for B, (bits, cut_want) in h["want"].items():
        side, cut = orc.merge_beam(g, first, size, cand, h["K"], int(B))
        assert "".join(str(int(b)) for b in side) == bits and cut == cut_want, B
    # B >= K^(M-1) = 4 is the exhaustive merge: the best leaf, cut 8
    side4, cut4 = orc.merge_beam(g, first, size, cand, h["K"], 4)
    sidex, cutx, _ = orc.merge_exhaustive(g, first, size, cand, h["K"], 1)
    assert cut4 == cutx == h["exhaustive_cut"] and np.array_equal(side4, sidex)


def test_merge_space_counts(orc):
    ex = GOLD["merge_space"]
    # 2K^L workers in the paper = K^L starting paths times the two orientations
    for L, wk in zip(ex["L"], ex["workers"]):
        assert 2 * ex["K"] ** L == wk
    g = synth.erdos_renyi(13, 0.4, 2)
    first, size = orc.partition(g.n, 4)
    cand = np.zeros((4, 2), np.uint32)
    cand[:, 1] = 1
    _, _, leaves = orc.merge_exhaustive(g, first, size, cand, K=2, L=2)
    assert 2 * leaves == 2 * ex["K"] ** 4


def test_ar_and_ef_examples():
    ex = GOLD["ar_example"]
    assert ex["alg"] / ex["opt"] == ex["ar"]
    assert 1 / (1 + np.exp(0.001 * (5.0 - 5.0))) == GOLD["efficiency_factor"]["ef_at_parity"]


def test_small_case_end_to_end_below_optimum(orc):
    """The tiny configuration: merged cut is a valid cut <= brute-force OPT."""
    g = synth.erdos_renyi(20, 0.5, 0)
    subs = orc.subgraphs(g, 2)
    batch = orc.Batch(subs)
    vals, arg, gb, bb = orc.grid_search(batch)
    K = 4
    cand = []
    for s, gg, b in zip(subs, gb, bb):
        st = orc.simulate(s, [gg], [b])
        z, _ = orc.topk(s.n, st, K)
        cand.append(z)
    first = [s.first for s in subs]
    size = [s.n for s in subs]
    side, cut, _ = orc.merge_exhaustive(g, first, size, np.array(cand), K, 1)
    opt, _ = orc.bruteforce_maxcut(orc.Subgraph(0, g.n, g.eu, g.ev, g.ew))
    assert cut == orc.cutval(g, side) <= opt
    assert cut >= 0.8 * opt


# ------------------------------------------------------------------ angle search
def test_weight_scaled_grid_undoes_a_uniform_weight(orc):
    """C_w = w C_1 for a graph whose edges all weigh w, so exp(-i (gamma / w)
    C_w) = exp(-i gamma C_1): the plain form's grid (gamma axis divided by the
    mean edge weight) on the weight-w graph must give, point for point, the
    unscaled grid's <C> on the unit-weight graph times w, and pick the same
    grid point; mixed weights get the divisor W / |E|."""
    g1 = synth.erdos_renyi(9, 0.5, 4)
    for w in (3, 7):
        gw = synth.from_edges(g1.n, np.stack([g1.eu, g1.ev], 1), np.full(len(g1.eu), w))
        v1, a1, ga1, _ = orc.grid_search(orc.Batch([sub_of(g1, orc)]), 8)
        vw, aw, gaw, _ = orc.grid_search(orc.Batch([sub_of(gw, orc)]), 8, weight_scaled=True)
        np.testing.assert_allclose(vw, w * v1, rtol=1e-12, atol=1e-12)
        assert aw[0] == a1[0] and gaw[0] == pytest.approx(ga1[0] / w)
        # unit weights: the scaled grid is the unscaled one
        vs, _, _, _ = orc.grid_search(orc.Batch([sub_of(g1, orc)]), 8, weight_scaled=True)
        np.testing.assert_array_equal(vs, v1)
    gm = synth.from_edges(3, [(0, 1), (1, 2)], [2, 7])
    assert orc.grid_scale(sub_of(gm, orc)) == 4.5
    assert orc.grid_scale(sub_of(synth.from_edges(3, []), orc)) == 1.0


def test_interp_and_canonicalize(orc):
    g2, b2 = orc.interp(np.array([[0.6]]), np.array([[-0.3]]))
    assert np.allclose(g2, [[0.6, 0.6]]) and np.allclose(b2, [[-0.3, -0.3]])
    g3, b3 = orc.interp(np.array([[0.2, 0.8]]), np.array([[0.5, 0.1]]))
    assert np.allclose(g3, [[0.2, 0.5, 0.8]]) and np.allclose(b3, [[0.5, 0.3, 0.1]])
    g = synth.erdos_renyi(9, 0.5, 2, wmax=3)
    s = sub_of(g, orc)
    gam, bet = np.array([4.0, -2.5]), np.array([1.2, -0.9])
    cg, cb = orc.canonicalize(gam, bet)
    assert 0 <= cg[0] <= np.pi and np.all(np.abs(cb) <= np.pi / 4)
    e1 = orc.expect_state(s, orc.simulate(s, gam, bet))
    e2 = orc.expect_state(s, orc.simulate(s, cg, cb))
    assert abs(e1 - e2) < 1e-10


def test_adam_improves_on_grid(orc):
    g = synth.erdos_renyi(40, 0.3, 1, wmax=10)
    subs = orc.subgraphs(g, 4)
    batch = orc.Batch(subs)
    vals, arg, gb, bb = orc.grid_search(batch, points=8)
    gf, bf, final = orc.adam_optimize(batch, gb[:, None], bb[:, None], orc.AdamConfig(steps=16))
    assert np.all(final >= vals.max(axis=1) - 1e-9)
