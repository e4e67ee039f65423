"""Split-precision tensor-core mixer (paraqaoa_simulate_tc) against the FP64
oracle and against the FP32 butterfly path, through the C ABI.

Error model (stated, not only bounded). Each FP32 operand is split into two
16-bit parts and the lo x lo product is dropped, so one mixer block commits
a relative error of about 2^-16 for BF16 parts (8 significant bits each) and
about 2^-22 for FP16 parts (11 bits each, on amplitudes scaled per block by a
power of two that brings a spread-out state's amplitudes near 1 and keeps
every amplitude below 2^15, so that the lo parts stay normal and nothing
overflows), plus FP32 accumulation. A depth-p circuit
applies ceil(n / k) blocks per layer. Bounds used below, per circuit:
FP16 split: amplitude max error <= 1e-5 and |d<C>| / W <= 1e-5 (the FP32
path's own tolerance); BF16 split: max error <= 2e-3 max|psi| and
|d<C>| / W <= 2e-3. The measured errors are printed (pytest -s) and listed
in the design notes.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi
    ctx = _capi.paraqaoa_create(0)
    yield _capi, ctx
    _capi.paraqaoa_destroy(ctx)


def _case(capi, orc, sizes, p, seed, wmax=10, p_edge=0.45):
    nv = int(sum(sizes) - (len(sizes) - 1))
    g = synth.erdos_renyi(nv, p_edge, seed, wmax=wmax)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    first, size = orc.partition(g.n, len(sizes), 2, sizes)
    subs = [orc.get_subgraph(g, int(f), int(s)) for f, s in zip(first, size)]
    gam, bet = synth.random_angles(len(sizes), p, 500 + seed)
    return part, subs, gam, bet


@pytest.mark.parametrize("precision,k", [(1, 7), (1, 6), (1, 5), (0, 7)])
def test_tc_mixer_against_oracle(api, orc, precision, k):
    capi, ctx = api
    sizes = [12, 13, 16, 17]
    p = 2
    part, subs, gam, bet = _case(capi, orc, sizes, p, 3 + k)
    try:
        ids = np.arange(len(sizes), dtype=np.int32)
        capi.paraqaoa_simulate_tc(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE,
                                  precision, k)
        ex = capi.paraqaoa_expect(ctx, len(ids))
        states = [capi.paraqaoa_state(ctx, i, s.n) for i, s in enumerate(subs)]
        # the FP32 butterfly path on the same instances
        capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
        ex32 = capi.paraqaoa_expect(ctx, len(ids))
        st32 = [capi.paraqaoa_state(ctx, i, s.n) for i, s in enumerate(subs)]
    finally:
        capi.paraqaoa_part_free(part)
    name = "FP16" if precision == 1 else "BF16"
    for i, s in enumerate(subs):
        ref = orc.simulate(s, gam[i], bet[i])
        W = s.total_weight
        err = float(np.max(np.abs(states[i] - ref)))
        l2 = float(np.linalg.norm(states[i] - ref))
        dex = abs(ex[i] - orc.expect_state(s, ref)) / W
        err32 = float(np.max(np.abs(st32[i] - ref)))
        dex32 = abs(ex32[i] - orc.expect_state(s, ref)) / W
        print(f"{name} k={k} n={s.n}: max|dpsi| {err:.2e} (fp32 path {err32:.2e}), ||dpsi||2 {l2:.2e}, "
              f"|d<C>|/W {dex:.2e} (fp32 path {dex32:.2e})")
        if precision == 1:
            assert err <= 1e-5 and dex <= 1e-5, (s.n, err, dex)
        else:
            assert err <= 2e-3 * np.max(np.abs(ref)) and dex <= 2e-3, (s.n, err, dex)


def test_tc_mixer_p3_and_repeated_calls(api, orc):
    """Depth 3 on a 20-qubit part (three mixer blocks of 7, 7, 6 per layer),
    twice in a row: identical results (fixed summation order)."""
    capi, ctx = api
    sizes = [20, 14]
    part, subs, gam, bet = _case(capi, orc, sizes, 3, 11, wmax=1, p_edge=0.3)
    try:
        ids = np.arange(2, dtype=np.int32)
        out = []
        for _ in range(2):
            capi.paraqaoa_simulate_tc(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT, capi.TC_FP16, 7)
            out.append(capi.paraqaoa_expect(ctx, 2))
    finally:
        capi.paraqaoa_part_free(part)
    assert np.array_equal(out[0], out[1])
    for i, s in enumerate(subs):
        ref = orc.simulate(s, gam[i], bet[i])
        assert abs(out[0][i] - orc.expect_state(s, ref)) / s.total_weight <= 1e-5


def test_tc_mixer_rejects_small_parts(api, orc):
    capi, ctx = api
    part, subs, gam, bet = _case(capi, orc, [11, 13], 1, 2)
    try:
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_simulate_tc(ctx, part, np.arange(2, dtype=np.int32), 1, gam, bet)
    finally:
        capi.paraqaoa_part_free(part)


@pytest.mark.parametrize("precision", [1, 0])
def test_tc_mixer_growth_at_quarter_pi(api, orc, precision):
    """beta = pi/4 (mu = -1: every gauge butterfly grows the norm by sqrt 2,
    the most a layer can) on parts of 20..24 qubits at p = 2 and 3: every
    amplitude finite, and within the split's tolerance of the FP32 path on
    4096 sampled amplitudes plus <C> (the FP16 scale of each block is lowered
    by the growth of the qubits mixed before it)."""
    capi, ctx = api
    sizes = [20, 22, 24]
    for p in (2, 3):
        part, subs, gam, _ = _case(capi, orc, sizes, p, 40 + p, p_edge=0.25)
        bet = np.full((len(sizes), p), np.pi / 4)
        try:
            ids = np.arange(len(sizes), dtype=np.int32)
            capi.paraqaoa_simulate_tc(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE,
                                      precision, 7)
            ex = capi.paraqaoa_expect(ctx, len(ids))
            st = [capi.paraqaoa_state(ctx, i, s.n) for i, s in enumerate(subs)]
            capi.paraqaoa_simulate_batch(ctx, part, ids, p, gam, bet, capi.SIM_EXPECT | capi.SIM_KEEP_STATE)
            ex32 = capi.paraqaoa_expect(ctx, len(ids))
            rng = np.random.default_rng(p)
            for i, s in enumerate(subs):
                ours = st[i]
                assert np.all(np.isfinite(ours.view(np.float32))), (p, s.n)
                ref = capi.paraqaoa_state(ctx, i, s.n)
                idx = rng.integers(0, 1 << s.n, 4096)
                err = float(np.max(np.abs(ours[idx] - ref[idx])))
                dex = abs(ex[i] - ex32[i]) / s.total_weight
                amax = float(np.max(np.abs(ref)))
                print(f"{'FP16' if precision else 'BF16'} beta=pi/4 p={p} n={s.n}: max|dpsi| {err:.2e}, "
                      f"|d<C>|/W {dex:.2e}")
                if precision == 1:
                    assert err <= 1e-5 and dex <= 1e-5, (p, s.n, err, dex)
                else:
                    assert err <= 2e-3 * amax and dex <= 2e-3, (p, s.n, err, dex)
            del st
        finally:
            capi.paraqaoa_part_free(part)


def test_tc_mixer_wait_limit_gives_timeout_and_context_survives(api, orc):
    """A wait limit of 0 makes the mixer's wait for its tensor-core products
    give up before its first poll: the call returns PARAQAOA_E_TIMEOUT (the
    kernel lets the products already issued finish before it frees its
    tensor memory), and with the default limit restored the same context
    gives the results of a fresh run."""
    capi, ctx = api
    part, subs, gam, bet = _case(capi, orc, [14, 16], 2, 9)
    try:
        ids = np.arange(2, dtype=np.int32)
        capi.paraqaoa_simulate_tc(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT, capi.TC_FP16, 7)
        before = capi.paraqaoa_expect(ctx, 2)
        capi.paraqaoa_set_wait_limit(ctx, 0)
        try:
            with pytest.raises(capi.ParaQAOAError) as e:
                capi.paraqaoa_simulate_tc(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT, capi.TC_FP16, 7)
            assert e.value.code == capi.E_TIMEOUT
        finally:
            capi.paraqaoa_set_wait_limit(ctx, 200_000_000)
        capi.paraqaoa_simulate_tc(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT, capi.TC_FP16, 7)
        assert np.array_equal(capi.paraqaoa_expect(ctx, 2), before)
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_set_wait_limit(ctx, -1)
    finally:
        capi.paraqaoa_part_free(part)
