"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (stated for the floating-point results): amplitude max error
<= 1e-5 and |<C>_gpu - <C>_oracle| / W <= 1e-5. Integer results (cut tables,
partitions, merged cuts) must match exactly.
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
EXP_TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi
    ctx = _capi.paraqaoa_create(0)
    yield _capi, ctx
    _capi.paraqaoa_destroy(ctx)


def chain_graph(sizes, p_edge, seed, wmax):
    """A graph whose SIZES partition has parts of exactly the given sizes."""
    nv = int(sum(sizes) - (len(sizes) - 1))
    return synth.erdos_renyi(nv, p_edge, seed, wmax=wmax)


def oracle_parts(orc, g, sizes):
    first, size = orc.partition(g.n, len(sizes), 2, sizes)
    return [orc.get_subgraph(g, int(f), int(s)) for f, s in zip(first, size)]


def test_cut_table_bit_exact(api, orc):
    capi, ctx = api
    sizes = [2, 2, 5, 10, 13, 14, 15, 17, 20]
    g = chain_graph(sizes, 0.4, 1, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        for i, s in enumerate(subs):
            ours = capi.paraqaoa_cut_table(ctx, part, i, s.n)
            ref = orc.cut_table(s)
            assert np.array_equal(ours.astype(np.int64), ref), f"part {i} (n={s.n})"
    finally:
        capi.paraqaoa_part_free(part)


def _state_case(capi, ctx, orc, sizes, p, seed, wmax=10, p_edge=0.45):
    g = chain_graph(sizes, p_edge, seed, wmax)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), p, 1000 + seed)
        capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex = capi.paraqaoa_expect(ctx, len(ids))
        for i, s in enumerate(subs):
            ref = orc.simulate(s, gam[i], bet[i])
            ours = capi.paraqaoa_state(ctx, i, s.n)
            err = np.max(np.abs(ours.astype(np.complex128) - ref))
            assert err <= AMP_TOL, f"n={s.n} p={p}: amplitude error {err}"
            W = max(s.total_weight, 1)
            e_ref = orc.expect_state(s, ref)
            assert abs(ex[i] - e_ref) / W <= EXP_TOL, f"n={s.n} p={p}: <C> {ex[i]} vs {e_ref}"
        # expectation-only run gives the same <C> without keeping states
        capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT)
        ex2 = capi.paraqaoa_expect(ctx, len(ids))
        assert np.max(np.abs(ex2 - ex)) <= 1e-9 * max(1.0, np.max(np.abs(ex)))
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_state_parity_small_and_onchip(api, orc, p):
    """n = 2..14: tiny and whole-state-on-chip kernels, mixed in one batch."""
    capi, ctx = api
    _state_case(capi, ctx, orc, [2, 3, 5, 8, 9, 10, 11, 12, 13, 14], p, seed=p)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_state_parity_streaming(api, orc, p):
    """n = 15..21: HBM layer passes (two qubit groups), mixed sizes in one batch."""
    capi, ctx = api
    _state_case(capi, ctx, orc, [15, 16, 17, 19, 21], p, seed=10 + p)


def test_state_parity_three_groups(api, orc):
    """n = 22 and 24: n = 24 needs a third qubit group (2p + 1 passes)."""
    capi, ctx = api
    _state_case(capi, ctx, orc, [22, 24], 2, seed=21, p_edge=0.3)


def test_unit_weight_and_edgeless_parts(api, orc):
    capi, ctx = api
    _state_case(capi, ctx, orc, [4, 12, 16], 2, seed=5, wmax=1, p_edge=0.5)
    _state_case(capi, ctx, orc, [6, 11, 15], 1, seed=6, wmax=1, p_edge=0.0)


def test_extreme_angles(api, orc):
    """beta near pi/4 and pi/2 exercise both mixer factorisations."""
    capi, ctx = api
    sizes = [9, 12, 16]
    g = chain_graph(sizes, 0.5, 3, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(3, dtype=np.int32)
        for b in [np.pi / 4, np.pi / 4 + 1e-7, np.pi / 2, -1.2, 0.0]:
            gam = np.full((3, 2), 0.7)
            bet = np.full((3, 2), b)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
            ex = capi.paraqaoa_expect(ctx, 3)
            for i, s in enumerate(subs):
                ref = orc.simulate(s, gam[i], bet[i])
                assert np.max(np.abs(capi.paraqaoa_state(ctx, i, s.n) - ref)) <= AMP_TOL
                assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL
    finally:
        capi.paraqaoa_part_free(part)


def _check_topk(orc, s, state_ref, z, pr, K):
    """Exact ids where the oracle's K-th/(K+1)-th gap is clear; otherwise every
    pick must be within 1e-5 max P of the oracle's K-th probability."""
    probs = np.abs(state_ref) ** 2
    half = 1 << (s.n - 1)
    cand = np.arange(half)
    order = np.lexsort((cand, -probs[:half]))
    oz = cand[order]
    pmax = probs.max()
    kth = probs[oz[K - 1]]
    nxt = probs[oz[K]] if K < half else -1.0
    assert np.all(z < half)
    assert len(set(z.tolist())) == K
    if kth - nxt > 1e-5 * pmax:
        assert set(z.tolist()) == set(oz[:K].tolist())
    else:
        assert np.all(probs[z] >= kth - 1e-5 * pmax)
    assert np.all(np.diff(pr) <= 0)
    assert np.max(np.abs(pr - probs[z])) <= 1e-5 * pmax


@pytest.mark.parametrize("K", [1, 4, 16, 32])
def test_topk_parity(api, orc, K):
    capi, ctx = api
    sizes = [7, 11, 14, 16, 18]
    g = chain_graph(sizes, 0.5, 7, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 2, 77)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_KEEP_STATE)
        z, pr = capi.paraqaoa_topk(ctx, len(ids), K)
        for i, s in enumerate(subs):
            _check_topk(orc, s, orc.simulate(s, gam[i], bet[i]), z[i], pr[i], K)
        # raw mode ranks both halves: every pick is at least as likely as the
        # oracle's K-th over all z, up to the tolerance
        zr, prr = capi.paraqaoa_topk(ctx, len(ids), K, capi.TOPK_RAW)
        for i, s in enumerate(subs):
            probs = np.abs(orc.simulate(s, gam[i], bet[i])) ** 2
            kth = np.sort(probs)[::-1][K - 1]
            assert len(set(zr[i].tolist())) == K
            assert np.all(probs[zr[i]] >= kth - 1e-5 * probs.max())
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_merge_exhaustive_parity(api, orc, seed):
    capi, ctx = api
    g = synth.erdos_renyi(40, 0.25, seed, wmax=5)
    G = capi.Graph.of(g)
    M, K = 4, 4
    part = capi.paraqaoa_partition(G, M)
    try:
        first, size, _, _ = capi.paraqaoa_part_info(part)
        rng = np.random.default_rng(seed)
        cand = np.array([rng.integers(0, 1 << int(s), K) for s in size], dtype=np.uint32)
        ref_side, ref_cut, _ = orc.merge_exhaustive(g, first, size, cand, K, 1)
        for L in (1, 2, 3, 4):
            side, cut = capi.paraqaoa_merge(ctx, G, part, cand, K, L, 0)
            assert cut == ref_cut and np.array_equal(side, ref_side)
            assert orc.cutval(g, side) == cut
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("beam", [1, 3, 16, 64])
def test_merge_beam_parity(api, orc, beam):
    capi, ctx = api
    g = synth.erdos_renyi(120, 0.1, 4, wmax=10)
    G = capi.Graph.of(g)
    M, K = 7, 8
    part = capi.paraqaoa_partition(G, M)
    try:
        first, size, _, _ = capi.paraqaoa_part_info(part)
        rng = np.random.default_rng(beam)
        cand = np.array([rng.integers(0, 1 << int(s), K) for s in size], dtype=np.uint32)
        ref_side, ref_cut = orc.merge_beam(g, first, size, cand, K, beam)
        side, cut = capi.paraqaoa_merge(ctx, G, part, cand, K, 1, beam)
        assert cut == ref_cut and np.array_equal(side, ref_side)
        assert orc.cutval(g, side) == cut
    finally:
        capi.paraqaoa_part_free(part)


def test_merge_beam_hand_worked_ties(api):
    """The hand-worked beam case of the oracle pins (ties planted at levels
    0 and 2, a complemented candidate at level 1): B = 1 and B = 2 give the
    assignments worked out by hand, B = 4 the exhaustive optimum."""
    capi, ctx = api
    h = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "beam_hand_case.json")))
    g = synth.from_edges(h["num_vertices"], h["edges"], h["weights"])
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, h["M"])
    try:
        cand = np.array(h["candidates"], np.uint32)
        for B, (bits, cut_want) in list(h["want"].items()) + [("4", (None, h["exhaustive_cut"]))]:
            side, cut = capi.paraqaoa_merge(ctx, G, part, cand, h["K"], 1, int(B))
            assert cut == cut_want, B
            if bits is not None:
                assert "".join(str(int(b)) for b in side) == bits, B
        side_x, cut_x = capi.paraqaoa_merge(ctx, G, part, cand, h["K"], 1, 0)
        assert cut_x == h["exhaustive_cut"] and np.array_equal(side_x, side)
    finally:
        capi.paraqaoa_part_free(part)


def test_merge_beam_16k_vertex_scale(api, orc):
    """The merge of the 16,000-vertex workload: G(16000, 0.01), unit weights,
    640 parts of 25-26 vertices, K = 32 seeded candidates per part, beam 64
    (500-word side bitsets, 640 levels): cut and assignment bit-exact
    against the oracle's beam merge."""
    capi, ctx = api
    g = synth.erdos_renyi(16000, 0.01, 0, wmax=1)
    G = capi.Graph.of(g)
    M, K, B = 640, 32, 64
    part = capi.paraqaoa_partition(G, M)
    try:
        first, size, _, _ = capi.paraqaoa_part_info(part)
        assert set(size.tolist()) == {25, 26}
        rng = np.random.default_rng(16000)
        cand = np.array([rng.integers(0, 1 << int(s), K) for s in size], dtype=np.uint32)
        side, cut = capi.paraqaoa_merge(ctx, G, part, cand, K, 1, B)
        oside, ocut = orc.merge_beam(g, first, size, cand, K, B)
        assert cut == ocut and np.array_equal(side, oside)
        assert orc.cutval(g, side) == cut
    finally:
        capi.paraqaoa_part_free(part)


def test_grid_search_parity_small_config(api, orc):
    """Tiny configuration: G(20, 0.5), unit weights, 2 parts, 16 x 16 grid."""
    capi, ctx = api
    g = synth.erdos_renyi(20, 0.5, 0)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 2)
    try:
        subs = orc.subgraphs(g, 2)
        ids = np.arange(2, dtype=np.int32)
        gg, bb, best, vals = capi.paraqaoa_grid_search(ctx, part, ids, 16, want_values=True)
        ovals, oarg, og, ob = orc.grid_search(orc.Batch(subs), 16)
        for i, s in enumerate(subs):
            W = s.total_weight
            assert np.max(np.abs(vals[i] - ovals[i])) / W <= EXP_TOL
            # the GPU's pick is a maximum of the oracle's values within tolerance
            k = int(np.argmax(vals[i]))
            assert ovals[i, k] >= ovals[i].max() - 2 * EXP_TOL * W
            assert abs(best[i] - vals[i, k]) < 1e-12
    finally:
        capi.paraqaoa_part_free(part)


def test_optimize_parity(api, orc):
    capi, ctx = api
    g = synth.erdos_renyi(60, 0.3, 2, wmax=10)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 4)
    try:
        subs = orc.subgraphs(g, 4)
        batch = orc.Batch(subs)
        ids = np.arange(4, dtype=np.int32)
        g0, b0, _, _ = capi.paraqaoa_grid_search(ctx, part, ids, 8)
        g2, b2 = orc.interp(g0[:, None], b0[:, None])
        cfg = orc.AdamConfig(steps=12, lr=0.02, h=1e-3)
        og, ob, oval = orc.adam_optimize(batch, g2, b2, cfg)
        gg, bb, val = capi.paraqaoa_optimize(ctx, part, ids, 2, g2, b2, cfg.steps, cfg.lr, cfg.h)
        at_ours = orc.expect_batch(batch, ids, gg, bb)
        W = np.array([s.total_weight for s in subs], float)
        assert np.all(np.abs(val - at_ours) / W <= EXP_TOL)
        assert np.all(val >= oval - 1e-4 * W)
    finally:
        capi.paraqaoa_part_free(part)


def test_small_config_end_to_end(api, orc):
    """G(20, 0.5): grid -> top-4 -> exhaustive merge; the merged cut equals the
    oracle's merge of the same candidates and is <= the brute-force optimum."""
    import paper_2603_26232_gb300 as pkg
    capi, ctx = api
    g = synth.erdos_renyi(20, 0.5, 0)
    solver = pkg.Solver()
    try:
        res = solver.solve(g, pkg.SolveConfig(M=2, K=4, p=1, grid_points=16))
    finally:
        solver.close()
    first, size = orc.partition(20, 2)
    side, cut, _ = orc.merge_exhaustive(g, first, size, res.cand, 4, 1)
    assert res.cut == cut and np.array_equal(res.side, side)
    assert orc.cutval(g, res.side) == res.cut
    opt, _ = orc.bruteforce_maxcut(orc.Subgraph(0, g.n, g.eu, g.ev, g.ew))
    assert res.cut <= opt and res.cut >= 0.8 * opt


def test_paper_scale_config_full_size(api, orc):
    """G(400, 0.1), weights 1..10, 21 parts of 20 qubits, p = 2 at fixed
    angles, top-16, beam 256: every <C> and top-16 list against the oracle,
    and the merged cut equal to the oracle's merge of the same lists."""
    capi, ctx = api
    g = synth.erdos_renyi(400, 0.1, 0, wmax=10)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 21)
    try:
        subs = orc.subgraphs(g, 21)
        ids = np.arange(21, dtype=np.int32)
        gam, bet = synth.random_angles(21, 2, 400)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex = capi.paraqaoa_expect(ctx, 21)
        z, pr = capi.paraqaoa_topk(ctx, 21, 16)
        oex = orc.expect_batch(orc.Batch(subs), ids, gam, bet)
        W = np.array([s.total_weight for s in subs], float)
        assert np.all(np.abs(ex - oex) / W <= EXP_TOL)
        for i in (0, 10, 20):
            _check_topk(orc, subs[i], orc.simulate(subs[i], gam[i], bet[i]), z[i], pr[i], 16)
        first, size = orc.partition(400, 21)
        oside, ocut = orc.merge_beam(g, first, size, z, 16, 256)
        side, cut = capi.paraqaoa_merge(ctx, G, part, z, 16, 1, 256)
        assert cut == ocut and np.array_equal(side, oside)
    finally:
        capi.paraqaoa_part_free(part)


def test_error_codes(api):
    capi, ctx = api
    g = synth.erdos_renyi(30, 0.3, 1)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 2)
    try:
        ids = np.zeros(1, np.int32)
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_simulate_batch(ctx, part, np.array([5], np.int32), 1, [0.1], [0.1])
        assert e.value.code == capi.E_INVAL
        capi.paraqaoa_simulate_batch(ctx, part, ids, 1, [0.1], [0.1], capi.SIM_EXPECT)
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_topk(ctx, 1, 4)  # states were not kept
        assert e.value.code == capi.E_NO_RESULT
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_expect(ctx, 2)  # count mismatch
        assert e.value.code == capi.E_NO_RESULT
        capi.paraqaoa_simulate_batch(ctx, part, ids, 1, [0.1], [0.1], capi.SIM_KEEP_STATE)
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_topk(ctx, 1, 33)
    finally:
        capi.paraqaoa_part_free(part)
    # admission: a budget far below one 20-qubit state is refused
    small = capi.paraqaoa_create(0, 1 << 20)
    try:
        g2 = synth.erdos_renyi(40, 0.2, 1)
        p2 = capi.paraqaoa_partition(capi.Graph.of(g2), 2)
        try:
            with pytest.raises(capi.ParaQAOAError) as e:
                capi.paraqaoa_simulate_batch(small, p2, np.array([0], np.int32), 1, [0.1], [0.1])
            assert e.value.code == capi.E_ADMISSION
        finally:
            capi.paraqaoa_part_free(p2)
    finally:
        capi.paraqaoa_destroy(small)
    # a part heavier than the phase table is refused
    heavy = synth.erdos_renyi(12, 0.9, 1, wmax=200)
    ph = capi.paraqaoa_partition(capi.Graph.of(heavy), 1)
    try:
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_simulate_batch(ctx, ph, ids, 1, [0.1], [0.1])
        assert e.value.code == capi.E_INVAL
    finally:
        capi.paraqaoa_part_free(ph)


def test_autotune_choices_keep_parity(api, orc):
    """The autotuner picks a tile size and contiguous run per qubit count; the
    tuned passes must still match the oracle."""
    capi, ctx = api
    sizes = [15, 18, 20, 22]
    g = chain_graph(sizes, 0.35, 31, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        choice = capi.paraqaoa_autotune(ctx, part, 2)
        for n in sizes:
            tb, rb, cm, sp, tp = choice[n]
            assert (tb, rb) in ((12, 5), (12, 4), (13, 5), (13, 4), (14, 4)) and cm in (2, 3, 4) and sp in (0, 1, 2, 3)
            assert 0 <= tp <= 4
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 2, 99)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex = capi.paraqaoa_expect(ctx, len(ids))
        for i, s in enumerate(subs):
            ref = orc.simulate(s, gam[i], bet[i])
            assert np.max(np.abs(capi.paraqaoa_state(ctx, i, s.n) - ref)) <= AMP_TOL
            assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("tb,rb,split,tpc", [(12, 5, 0, 0), (12, 4, 0, 0), (13, 5, 0, 0), (12, 5, 1, 0), (12, 4, 1, 0),
                                             (13, 5, 1, 0), (12, 4, 0, 3), (12, 4, 1, 2), (12, 5, 0, 2),
                                             (12, 5, 1, 3), (13, 5, 0, 1), (13, 5, 1, 2), (13, 4, 0, 0),
                                             (13, 4, 0, 2), (13, 4, 1, 1), (14, 4, 0, 0), (14, 4, 0, 3),
                                             (14, 4, 1, 0), (12, 4, 2, 3), (12, 5, 3, 0), (13, 5, 2, 2),
                                             (13, 4, 3, 1), (14, 4, 2, 0)])
def test_every_schedule_matches_oracle(api, orc, tb, rb, split, tpc):
    """Every tile shape in every schedule form (classic or split, low or high
    group first), one or several tiles per CTA, on parts of 15..24 qubits
    (two and three qubit groups), depth 3, states kept."""
    capi, ctx = api
    sizes = [15, 16, 19, 20, 21, 23, 24]
    g = chain_graph(sizes, 0.3, 40 + tb + rb + split + tpc, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        for n in sizes:
            capi.paraqaoa_set_schedule(ctx, n, tb, rb, 3, split, tpc)
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 3, 123 + split)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex = capi.paraqaoa_expect(ctx, len(ids))
        for i, s in enumerate(subs):
            ref = orc.simulate(s, gam[i], bet[i])
            assert np.max(np.abs(capi.paraqaoa_state(ctx, i, s.n) - ref)) <= AMP_TOL, (s.n,)
            assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL, (s.n,)
        # <C> without kept states takes the expect-only last pass
        capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
        ex2 = capi.paraqaoa_expect(ctx, len(ids))
        assert np.all(np.abs(ex2 - ex) <= 1e-9 * np.abs(ex))
    finally:
        for n in sizes:
            capi.paraqaoa_set_schedule(ctx, n, 12, 4, 3, 0)
        capi.paraqaoa_part_free(part)


def test_default_schedules_match_oracle(api, orc):
    """A fresh context's built-in schedules (no autotune, no set_schedule):
    2^13 x 32 registers, split and high group first, walking 8 tiles (16
    qubits: 2^12 x 16 walking 16), classic and high first for 21-24; depth 2,
    states kept."""
    capi, _ = api
    ctx = capi.paraqaoa_create(0)
    sizes = [15, 16, 17, 19, 20, 21, 23, 24]
    g = chain_graph(sizes, 0.3, 91, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 2, 92)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex = capi.paraqaoa_expect(ctx, len(ids))
        for i, s in enumerate(subs):
            ref = orc.simulate(s, gam[i], bet[i])
            assert np.max(np.abs(capi.paraqaoa_state(ctx, i, s.n) - ref)) <= AMP_TOL, (s.n,)
            assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL, (s.n,)
    finally:
        capi.paraqaoa_part_free(part)
        capi.paraqaoa_destroy(ctx)


def test_set_schedule_rejects_out_of_range(api):
    """Host-side validation of hand-set schedules: unknown shapes, runs, form
    bits, tiles per CTA above 2^4, split schedules that do not fit the part."""
    capi, ctx = api
    for args in [(20, 12, 3, 2, 0, 0), (20, 12, 4, 9, 0, 0), (20, 12, 4, 2, 4, 0), (20, 12, 4, 2, -1, 0),
                 (20, 12, 4, 2, 0, 5),
                 (20, 13, 5, 2, 0, 5), (8, 12, 4, 2, 0, 0), (20, 14, 5, 2, 0, 0), (20, 14, 4, 1, 0, 0),
                 (20, 13, 4, 0, 0, 0)]:
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_set_schedule(ctx, *args)
    capi.paraqaoa_set_schedule(ctx, 20, 12, 4, 2, 0, 4)   # the largest walk is accepted
    capi.paraqaoa_set_schedule(ctx, 20, 12, 4, 3, 0)


def test_large_parts_full_size(api, orc):
    """Parts of 25 and 26 qubits (the 16,000-vertex workload's sizes, 256 and
    512 MB complex64 states), p = 2, in the schedule the context uses by
    default there (2^13 x 32, split and high group first: three qubit groups,
    five passes, 8 tiles per CTA), the split 2^12 x 32 one, a classic 2^13
    one and two groups on the 2^14 x 16 tile: <C>, 4096 sampled amplitudes
    plus the top-32 entries, and the top-32 lists."""
    capi, ctx = api
    sizes = [25, 26]
    g = chain_graph(sizes, 0.15, 77, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), 2, capi.PART_SIZES, sizes)
    subs = oracle_parts(orc, g, sizes)
    gam, bet = synth.random_angles(2, 2, 2526)
    refs = [orc.simulate(s, gam[i], bet[i]) for i, s in enumerate(subs)]
    oex = [orc.expect_state(s, r) for s, r in zip(subs, refs)]
    rng = np.random.default_rng(5)
    try:
        # three groups in the split 2^12 x 32 schedule, a classic 2^13 one, and
        # two groups on the 2^14 x 16 tile (four register rounds in the low group)
        for sched in [(13, 5, 2, 3, 3), (12, 5, 2, 1, 2), (13, 5, 2, 0), (14, 4, 2, 0, 2)]:
            for n in sizes:
                capi.paraqaoa_set_schedule(ctx, n, *sched)
            ids = np.arange(2, dtype=np.int32)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
            ex = capi.paraqaoa_expect(ctx, 2)
            z, pr = capi.paraqaoa_topk(ctx, 2, 32)
            for i, s in enumerate(subs):
                assert abs(ex[i] - oex[i]) / s.total_weight <= EXP_TOL, (sched, s.n)
                ours = capi.paraqaoa_state(ctx, i, s.n)
                idx = np.concatenate([rng.integers(0, 1 << s.n, 4096), z[i].astype(np.int64)])
                assert np.max(np.abs(ours[idx] - refs[i][idx])) <= AMP_TOL, (sched, s.n)
                del ours
                _check_topk(orc, s, refs[i], z[i], pr[i], 32)
    finally:
        for n in sizes:
            capi.paraqaoa_set_schedule(ctx, n, 12, 4, 3, 0)
        capi.paraqaoa_part_free(part)


def test_optimize_graph_replay_matches_direct_launches(api):
    """With per-kernel profiling off, Adam steps 2.. replay one captured step
    as a CUDA graph; with profiling on, every step is launched directly. Both
    must give identical angles and <C> (the kernels are deterministic)."""
    capi, ctx = api
    g = synth.erdos_renyi(60, 0.3, 4, wmax=10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), 4)
    try:
        ids = np.arange(4, dtype=np.int32)
        g0, b0 = synth.random_angles(4, 2, 8)
        out = []
        for prof in (False, True):
            capi.paraqaoa_profile_enable(ctx, prof)
            out.append(capi.paraqaoa_optimize(ctx, part, ids, 2, g0, b0, 6))
        capi.paraqaoa_profile_enable(ctx, False)
    finally:
        capi.paraqaoa_part_free(part)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_profile_classes_mask(api):
    """With the event brackets restricted to the layer passes, every class
    still counts its launches and bytes, only the layer passes get device
    time, and the results equal those of an unprofiled run."""
    capi, ctx = api
    g = synth.erdos_renyi(60, 0.3, 5, wmax=10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), 3)
    try:
        ids = np.arange(3, dtype=np.int32)
        gam, bet = synth.random_angles(3, 2, 9)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)
        ref = capi.paraqaoa_expect(ctx, 3)
        capi.paraqaoa_profile_enable(ctx, True)
        capi.paraqaoa_profile_classes(ctx, 1 << capi.KCLASS_LAYER_PASS)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)
        ex = capi.paraqaoa_expect(ctx, 3)
        lp = capi.paraqaoa_profile_read(ctx, capi.KCLASS_LAYER_PASS)
        other = capi.paraqaoa_profile_read(ctx, capi.KCLASS_OTHER)
    finally:
        capi.paraqaoa_profile_enable(ctx, False)
        capi.paraqaoa_profile_classes(ctx, 0xFFFFFFFF)
        capi.paraqaoa_part_free(part)
    assert np.array_equal(ex, ref)
    assert lp[0] > 0 and lp[1] > 0 and lp[2] > 0
    assert other[0] > 0 and other[1] == 0.0


def test_size_classes_on_side_streams_match_serial(api, orc):
    """Uneven parts (9..22 qubits: tiny, on-chip and streamed classes) in one
    batch: with profiling off the size classes run concurrently on side
    streams, with profiling on they run in order on the context stream. The
    results must be identical, and match the oracle."""
    capi, ctx = api
    sizes = [9, 12, 14, 15, 17, 20, 22, 16, 13]
    g = chain_graph(sizes, 0.3, 66, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 3, 67)
        out = []
        for prof in (False, True):
            capi.paraqaoa_profile_enable(ctx, prof)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
            out.append(capi.paraqaoa_expect(ctx, len(ids)))
        capi.paraqaoa_profile_enable(ctx, False)
        assert np.array_equal(out[0], out[1])
        subs = oracle_parts(orc, g, sizes)
        oex = orc.expect_batch(orc.Batch(subs), ids, gam, bet)
        W = np.array([s.total_weight for s in subs], float)
        assert np.all(np.abs(out[0] - oex) / W <= EXP_TOL)
    finally:
        capi.paraqaoa_part_free(part)


def test_persistent_layer_passes_match_per_pass_launches(api, orc):
    """The persistent form (every pass of every size class of one tile shape
    in one launch over a work queue) on uneven parts of 9..24 qubits and two
    tile shapes: states and <C> bit-identical to the per-pass launches, and
    within the tolerances of the oracle."""
    capi, ctx = api
    sizes = [9, 13, 15, 16, 18, 20, 21, 22, 24, 17]
    g = chain_graph(sizes, 0.3, 303, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        for n, sc in {15: (12, 5, 2, 1, 1), 16: (12, 4, 2, 2, 2), 17: (12, 4, 2, 0, 0), 18: (12, 4, 3, 3, 1),
                      20: (12, 4, 2, 2, 3), 21: (13, 4, 2, 0, 2), 22: (13, 4, 2, 2, 1), 24: (13, 4, 2, 0, 0)}.items():
            capi.paraqaoa_set_schedule(ctx, n, *sc)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), 3, 304)
        out = []
        for persistent in (False, True):
            capi.paraqaoa_set_persistent(ctx, persistent)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
            ex = capi.paraqaoa_expect(ctx, len(ids))
            out.append((ex, [capi.paraqaoa_state(ctx, i, n) for i, n in enumerate(sizes)]))
            # repeated runs of one plan (the queue and counters are reset per run)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
            assert np.array_equal(capi.paraqaoa_expect(ctx, len(ids)), ex)
        assert np.array_equal(out[0][0], out[1][0])
        for a, b in zip(out[0][1], out[1][1]):
            assert np.array_equal(a, b)
        subs = oracle_parts(orc, g, sizes)
        for i, s in enumerate(subs):
            if s.n > 20:
                continue
            ref = orc.simulate(s, gam[i], bet[i])
            assert np.max(np.abs(out[1][1][i] - ref)) <= AMP_TOL, s.n
            assert abs(out[1][0][i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL, s.n
    finally:
        capi.paraqaoa_set_persistent(ctx, False)
        for n in (15, 16, 17, 18, 20, 21, 22, 24):
            capi.paraqaoa_set_schedule(ctx, n, 12, 4, 3, 0)
        capi.paraqaoa_part_free(part)


def test_persistent_adam_graph_replay_and_wait_timeout(api):
    """Adam steps replayed from one captured CUDA graph around the persistent
    launch give the per-pass launches' angles bit for bit. A wait limit of 0
    makes every queue wait give up at once: the results call returns
    PARAQAOA_E_TIMEOUT, and with the limit restored the context computes the
    earlier results again."""
    capi, ctx = api
    g = synth.erdos_renyi(70, 0.3, 71, wmax=10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), 4)
    try:
        ids = np.arange(4, dtype=np.int32)
        g0, b0 = synth.random_angles(4, 2, 72)
        out = []
        for persistent in (False, True):
            capi.paraqaoa_set_persistent(ctx, persistent)
            out.append(capi.paraqaoa_optimize(ctx, part, ids, 2, g0, b0, 5))
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, g0, b0, capi.SIM_EXPECT)
        ref = capi.paraqaoa_expect(ctx, 4)
        capi.paraqaoa_set_wait_limit(ctx, 0)
        try:
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, g0, b0, capi.SIM_EXPECT)
            with pytest.raises(capi.ParaQAOAError) as e:
                capi.paraqaoa_expect(ctx, 4)
            assert e.value.code == capi.E_TIMEOUT
        finally:
            capi.paraqaoa_set_wait_limit(ctx, 200_000_000)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, g0, b0, capi.SIM_EXPECT)
        assert np.array_equal(capi.paraqaoa_expect(ctx, 4), ref)
    finally:
        capi.paraqaoa_set_persistent(ctx, False)
        capi.paraqaoa_part_free(part)


def test_merge_fill_matches_paper_worker_split(api, orc):
    """The exhaustive merge's GPU walk started deeper than L (2^17 starting
    paths) against exactly K^L walkers and against the oracle's DFS: cut and
    assignment bit-exact for L = 1..3 on 12 parts (4096 paths), and the
    starting level each used."""
    capi, ctx = api
    g = synth.erdos_renyi(12 * 25 + 1, 0.1, 12, wmax=3)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 12)
    try:
        first, size, _, _ = capi.paraqaoa_part_info(part)
        rng = np.random.default_rng(12)
        cand = np.array([rng.integers(0, 1 << int(s), 2) for s in size], dtype=np.uint32)
        oside, ocut, leaves = orc.merge_exhaustive(g, first, size, cand, 2, 1)
        assert leaves == 4096
        for fill in (1, 0):
            capi.paraqaoa_set_merge_fill(ctx, fill)
            for L in (1, 2, 3):
                side, cut = capi.paraqaoa_merge(ctx, G, part, cand, 2, L, 0)
                assert cut == ocut and np.array_equal(side, oside), (fill, L)
                assert capi.paraqaoa_set_merge_fill(ctx, -1) == (12 if fill else L)
    finally:
        capi.paraqaoa_set_merge_fill(ctx, 1)
        capi.paraqaoa_part_free(part)


def test_merge_exhaustive_600_vertices_two_candidates(api, orc):
    """The paper's merge scale (600 vertices, 24 parts, K = 2: 2^24 paths)
    with a filled GPU walk: the same cut and assignment for L = 1, 2, 3, the
    cut is CutVal of the assignment, and no beam of width up to 4096 finds a
    larger cut."""
    capi, ctx = api
    g = synth.erdos_renyi(600, 0.1, 0, wmax=1)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, 24)
    try:
        _, size, _, _ = capi.paraqaoa_part_info(part)
        rng = np.random.default_rng(600)
        cand = np.array([rng.integers(0, 1 << int(s), 2) for s in size], dtype=np.uint32)
        res = [capi.paraqaoa_merge(ctx, G, part, cand, 2, L, 0) for L in (1, 2, 3)]
        for side, cut in res[1:]:
            assert cut == res[0][1] and np.array_equal(side, res[0][0])
        assert orc.cutval(g, res[0][0]) == res[0][1]
        for B in (16, 4096):
            _, cb = capi.paraqaoa_merge(ctx, G, part, cand, 2, 1, B)
            assert cb <= res[0][1]
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_halved_states_match_oracle(api, orc, p):
    """Halved states (PARAQAOA_SIM_HALVED: parts of >= 16 qubits keep z <
    2^(n-1), the top qubit's mixer pairs each z with its complement inside
    the low-group passes): the whole state read back, <C> and the canonical
    top-16 against the oracle, on parts of 16..22 qubits beside an on-chip
    part (simulated in full), with the 2^12 x 16 and 2^13 x 16 tiles."""
    capi, ctx = api
    sizes = [12, 16, 17, 19, 20, 21, 22]
    g = chain_graph(sizes, 0.35, 700 + p, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(len(sizes), dtype=np.int32)
        gam, bet = synth.random_angles(len(sizes), p, 710 + p)
        for sched in [(12, 4, 2, 0, 1), (13, 4, 2, 0, 0), (12, 4, 3, 0, 3)]:
            for n in (15, 16, 18, 19, 20, 21):  # halved parts of n vertices use n - 1's schedule
                capi.paraqaoa_set_schedule(ctx, n, *sched)
            flags = capi.SIM_EXPECT | capi.SIM_KEEP_STATE | capi.SIM_HALVED
            capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, flags)
            ex = capi.paraqaoa_expect(ctx, len(ids))
            z, pr = capi.paraqaoa_topk(ctx, len(ids), 16)
            for i, s in enumerate(subs):
                ref = orc.simulate(s, gam[i], bet[i])
                ours = capi.paraqaoa_state(ctx, i, s.n)
                assert np.max(np.abs(ours - ref)) <= AMP_TOL, (sched, s.n)
                assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL, (sched, s.n)
                _check_topk(orc, s, ref, z[i], pr[i], 16)
            with pytest.raises(capi.ParaQAOAError):
                capi.paraqaoa_topk(ctx, len(ids), 4, capi.TOPK_RAW)
            # <C> without kept states (the expect-only last pass) agrees
            capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_HALVED)
            ex2 = capi.paraqaoa_expect(ctx, len(ids))
            assert np.all(np.abs(ex2 - ex) <= 1e-9 * np.abs(ex)), sched
    finally:
        for n in (15, 16, 18, 19, 20, 21):
            capi.paraqaoa_set_schedule(ctx, n, 12, 4, 3, 0)
        capi.paraqaoa_part_free(part)


def test_halved_states_extreme_angles_and_full_size(api, orc):
    """Halved states at beta = +-pi/4 and pi/2 (both mixer factorisations)
    and a 24-qubit part (three qubit groups), against the oracle; and a
    26-qubit part against the full-state path (<C> and 4096 sampled
    amplitudes)."""
    capi, ctx = api
    sizes = [16, 18, 24]
    g = chain_graph(sizes, 0.3, 720, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    try:
        subs = oracle_parts(orc, g, sizes)
        ids = np.arange(3, dtype=np.int32)
        for b in [np.pi / 4, -np.pi / 4, np.pi / 2, 0.3]:
            gam = np.full((3, 2), 0.45)
            bet = np.full((3, 2), b)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet,
                                         capi.SIM_EXPECT | capi.SIM_KEEP_STATE | capi.SIM_HALVED)
            ex = capi.paraqaoa_expect(ctx, 3)
            for i, s in enumerate(subs):
                ref = orc.simulate(s, gam[i], bet[i])
                assert np.max(np.abs(capi.paraqaoa_state(ctx, i, s.n) - ref)) <= AMP_TOL, (b, s.n)
                assert abs(ex[i] - orc.expect_state(s, ref)) / s.total_weight <= EXP_TOL, (b, s.n)
    finally:
        capi.paraqaoa_part_free(part)
    g26 = synth.erdos_renyi(26, 0.2, 726, wmax=10)
    p26 = capi.paraqaoa_partition(capi.Graph.of(g26), 1)
    try:
        ids = np.zeros(1, np.int32)
        gam, bet = synth.random_angles(1, 2, 727)
        out = []
        for flags in (0, capi.SIM_HALVED):
            capi.paraqaoa_simulate_batch(ctx, p26, ids, 2, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE | flags)
            out.append((capi.paraqaoa_expect(ctx, 1)[0], capi.paraqaoa_state(ctx, 0, 26)))
        W = float(capi.paraqaoa_part_info(p26)[3][0])
        assert abs(out[0][0] - out[1][0]) / W <= EXP_TOL
        idx = np.random.default_rng(26).integers(0, 1 << 26, 4096)
        assert np.max(np.abs(out[0][1][idx] - out[1][1][idx])) <= AMP_TOL
    finally:
        capi.paraqaoa_part_free(p26)


def test_context_halved_setting_drives_the_angle_search(api, orc):
    """paraqaoa_set_halved: the grid search, Adam and the final top-K of a
    context that halves its states against a full-state context: every grid
    <C> within 1e-5 W, Adam's final <C> at its own angles within 1e-5 W of the
    oracle, and the tensor-core variant still simulating full states."""
    capi, ctx = api
    sizes = [16, 18, 20]
    g = chain_graph(sizes, 0.3, 730, 10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), 3, capi.PART_SIZES, sizes)
    hctx = capi.paraqaoa_create(0)
    try:
        capi.paraqaoa_set_halved(hctx, True)
        ids = np.arange(3, dtype=np.int32)
        subs = oracle_parts(orc, g, sizes)
        W = np.array([s.total_weight for s in subs], float)
        _, _, _, vf = capi.paraqaoa_grid_search(ctx, part, ids, 8, want_values=True)
        _, _, _, vh = capi.paraqaoa_grid_search(hctx, part, ids, 8, want_values=True)
        assert np.all(np.abs(vf - vh) <= EXP_TOL * W[:, None])
        g0, b0 = synth.random_angles(3, 2, 731)
        gg, bb, val = capi.paraqaoa_optimize(hctx, part, ids, 2, g0, b0, 4)
        oex = orc.expect_batch(orc.Batch(subs), ids, gg, bb)
        assert np.all(np.abs(val - oex) <= EXP_TOL * W)
        ex, z, pr = capi.paraqaoa_final_topk(hctx, part, ids, 2, gg, bb, 8)
        for i, s in enumerate(subs):
            _check_topk(orc, s, orc.simulate(s, gg[i], bb[i]), z[i], pr[i], 8)
        capi.paraqaoa_simulate_tc(hctx, part, ids, 2, gg, bb, capi.SIM_EXPECT | capi.SIM_KEEP_STATE, capi.TC_FP16, 7)
        assert np.all(np.abs(capi.paraqaoa_expect(hctx, 3) - oex) <= EXP_TOL * W)
        st = capi.paraqaoa_state(hctx, 2, 20)
        ref = orc.simulate(subs[2], gg[2], bb[2])
        assert np.max(np.abs(st - ref)) <= AMP_TOL
    finally:
        capi.paraqaoa_destroy(hctx)
        capi.paraqaoa_part_free(part)


def test_probe_streams_measures_plausible_bandwidth(api):
    """paraqaoa_probe_streams on 1 GiB buffers (past the 129 MB L2): write-only,
    read-only and copy bandwidth positive and finite, below the HBM3e nominal
    7.9 TB/s with margin for measurement, and not an order of magnitude below
    it (the half passes' ceilings are read from these)."""
    capi, _ = api
    w, r, c = capi.paraqaoa_probe_streams(0, 1 << 30)
    for v in (w, r, c):
        assert np.isfinite(v) and 1000.0 < v < 12000.0, (w, r, c)

