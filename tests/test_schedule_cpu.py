"""The layer-pass schedule (paraqaoa_schedule, host code of the C ABI) checked
on the CPU by replaying it symbolically: every pass's tile holds distinct
qubits of the state, every layer's mixer covers each qubit exactly once, the
phase of layer l comes after all of layer l-1's mixer and before any of
layer l's, and the pass count is 1 + p (G - 1) for G qubit groups.

The mixers of one layer act on different qubits and commute, so this order
is the circuit U_M(b_{p-1}) U_C(g_{p-1}) ... U_M(b_0) U_C(g_0) |+> of Sec. 2.2."""
import itertools

import pytest

from paper_2603_26232_gb300 import _capi as capi

SHAPES = [(12, 5), (12, 4), (13, 5), (13, 4), (14, 4)]


def _lay_off(tb, r, rho):
    """Register-bit offset of round rho of a classic pass: tb - r, tb - 2r, ...,
    then 0 for the last of ceil(tb / r) rounds."""
    full = -(-tb // r)
    return tb - (rho + 1) * r if rho + 1 < full else 0


def _rounds(pd, tb, r):
    """Register rounds a classic pass needs to reach its lowest mixed local bit."""
    k, full = 1, -(-tb // r)
    while k < full and pd["mix_lo"] < _lay_off(tb, r, k - 1):
        k += 1
    return k


def _tile_qubits(pd, tb):
    return [lb if lb < pd["c"] else pd["s"] + (lb - pd["c"]) for lb in range(tb)]


def _mixed_qubits(pd, tb, r):
    q = _tile_qubits(pd, tb)
    if pd["split"]:
        return set(q[: 2 * r])
    return set(q[pd["mix_lo"]:])


def _replay(n, p, tb, r, c_min, form, keep, expect):
    passes = capi.paraqaoa_schedule(n, p, tb, r, c_min, form, keep, expect)
    split, high_first = form & capi.SCHED_SPLIT, form & capi.SCHED_HIGH_FIRST
    full = set(range(n))
    mixed = [set() for _ in range(p)]
    phased = [False] * p
    groups = set()
    initialised = False
    for i, pd in enumerate(passes):
        tq = _tile_qubits(pd, tb)
        assert len(set(tq)) == tb and all(0 <= q < n for q in tq), (i, pd)
        assert pd["init"] == (1 if i == 0 else 0)
        assert pd["last"] == (1 if i == len(passes) - 1 else 0)
        if pd["c"] < tb:  # a high group carries at least c_min contiguous low qubits
            assert pd["c"] >= min(c_min, tb - 1) and not pd["split"]
        assert pd["split"] == (1 if split and pd["c"] == tb else 0)
        mq = _mixed_qubits(pd, tb, r)
        assert mq
        if not pd["split"]:
            # the rounds cover the mixed local bits [mix_lo, tb) and nothing
            # below; passes over a high group fit in at most three rounds
            k = _rounds(pd, tb, r)
            assert _lay_off(tb, r, k - 1) <= pd["mix_lo"] or k == -(-tb // r)
            if pd["c"] < tb:
                assert k <= 3, (n, tb, r, pd)
        groups.add(frozenset(mq))
        initialised = initialised or bool(pd["init"])
        assert initialised
        if pd["layerA"] >= 0:  # finish a mixer started by an earlier pass
            la = pd["layerA"]
            assert phased[la] and mixed[la] and not (mixed[la] & mq)
            mixed[la] |= mq
        if pd["layerP"] >= 0:
            lp = pd["layerP"]
            assert not phased[lp]
            assert lp == 0 or mixed[lp - 1] == full, "phase before the previous mixer is complete"
            assert all(phased[:lp])
            phased[lp] = True
        if pd["layerB"] >= 0:  # start a mixer on this pass's group, after its phase
            lb = pd["layerB"]
            assert phased[lb] and not mixed[lb]
            assert pd["layerP"] == lb
            mixed[lb] |= mq
        if i < len(passes) - 1:
            assert pd["store"] == 1 and pd["expect"] == 0
        else:
            assert pd["store"] == (1 if keep else 0) and pd["expect"] == (1 if expect else 0)
    assert all(phased) and all(m == full for m in mixed)
    # the groups partition the qubits
    assert sum(len(g) for g in groups) == n and set().union(*groups) == full
    assert len(passes) == 1 + p * (len(groups) - 1)
    return passes, len(groups)


@pytest.mark.parametrize("tb,r", SHAPES)
@pytest.mark.parametrize("form", [0, 1, 2, 3])
def test_schedules_replay_the_circuit(tb, r, form):
    for n, p, c_min, keep, expect in itertools.product(range(15, 31), (1, 2, 3, 4), (2, 3, 4), (0, 1), (0, 1)):
        if n < tb:
            continue
        _replay(n, p, tb, r, c_min, form, keep, expect)


def test_high_group_first_order():
    # n = 20 on 2^12 x 16: the write-only first pass and, at p = 2, the
    # read-only last pass mix the 8-qubit high group; the full pass between
    # them mixes the 12-qubit low group twice around the phase of layer 1
    passes, G = _replay(20, 2, 12, 4, 2, capi.SCHED_HIGH_FIRST, 0, 1)
    assert G == 2 and [pd["c"] for pd in passes] == [4, 12, 4]
    assert (passes[1]["layerA"], passes[1]["layerP"], passes[1]["layerB"]) == (0, 1, 1)
    # p = 1: the last pass is the low group's
    passes, _ = _replay(20, 1, 12, 4, 2, capi.SCHED_HIGH_FIRST, 0, 1)
    assert [pd["c"] for pd in passes] == [4, 12]
    # three groups: layer 0 runs 2, 1, 0 and layer 1 runs 0, 1, 2
    passes, G = _replay(26, 2, 12, 5, 2, capi.SCHED_SPLIT | capi.SCHED_HIGH_FIRST, 0, 1)
    assert G == 3 and [pd["s"] for pd in passes] == [18, 10, 12, 10, 18]
    # the same pass count as the low-group-first form
    for n, p in itertools.product((17, 20, 23, 26), (1, 2, 3)):
        assert len(_replay(n, p, 12, 4, 2, 2, 0, 1)[0]) == len(_replay(n, p, 12, 4, 2, 0, 0, 1)[0])


def test_pass_counts_of_the_measured_schedules():
    # two groups at n = 20 (12 + 8 qubits): p = 2 takes three passes
    passes, G = _replay(20, 2, 12, 4, 2, 0, 0, 1)
    assert G == 2 and len(passes) == 3
    assert [pd["c"] for pd in passes] == [12, 4, 12]
    # n = 26, split 2^12 x 32: 10 low qubits + two groups of 8 -> five passes at p = 2
    passes, G = _replay(26, 2, 12, 5, 2, 1, 0, 1)
    assert G == 3 and len(passes) == 5
    # n = 24 on the 2^13 tile: 13 + 11 qubits (2 contiguous carried), three passes
    passes, G = _replay(24, 2, 13, 5, 2, 0, 0, 1)
    assert G == 2 and passes[1]["c"] == 2
    # n = 26 on the 2^14 x 16 tile: 14 + 12 qubits (2 carried): two groups, three passes;
    # its low group takes four register rounds
    passes, G = _replay(26, 2, 14, 4, 2, 0, 0, 1)
    assert G == 2 and len(passes) == 3 and passes[1]["c"] == 2 and _rounds(passes[0], 14, 4) == 4
    # n = 22 on the 2^13 x 16 tile: 13 + 9 qubits, four carried (128-byte runs)
    passes, G = _replay(22, 2, 13, 4, 2, 0, 0, 1)
    assert G == 2 and passes[1]["c"] == 4 and _rounds(passes[1], 13, 4) == 3


def test_schedule_rejects_invalid_arguments():
    for args in [(20, 2, 12, 3, 2, 0), (20, 2, 14, 5, 2, 0), (11, 1, 12, 4, 2, 0), (20, 0, 12, 4, 2, 0),
                 (20, 17, 12, 4, 2, 0), (31, 1, 12, 4, 2, 0), (20, 1, 12, 4, 9, 0), (20, 1, 12, 4, 2, 4),
                 (20, 1, 12, 4, 2, -1)]:
        with pytest.raises(capi.ParaQAOAError):
            capi.paraqaoa_schedule(*args)
