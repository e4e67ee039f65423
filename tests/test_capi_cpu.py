"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-only partition (Alg. 1 + GetSubgraph) matches
the oracle bit for bit."""
import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def capi():
    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi
    _capi.load()
    return _capi


def test_exports_every_declared_symbol(capi):
    lib = ctypes.CDLL(capi.LIB_PATH)
    names = capi.declared_symbols()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_names_every_code(capi):
    codes = [capi.OK, capi.E_INVAL, capi.E_TOO_MANY_QUBITS, capi.E_ADMISSION, capi.E_NOMEM,
             capi.E_SEARCH_TOO_LARGE, capi.E_CUDA, capi.E_TIMEOUT, capi.E_NO_RESULT]
    msgs = [capi.strerror(c) for c in codes]
    assert len(set(msgs)) == len(msgs)
    assert capi.strerror(-99) == "unknown error"


@pytest.mark.parametrize("nv,M,mode,sizes", [
    (20, 2, 0, None), (400, 21, 0, None), (10, 3, 1, None), (97, 7, 1, None), (60, 5, 0, None),
    (300, None, 2, "uneven"),
])
def test_partition_matches_oracle(capi, orc, nv, M, mode, sizes):
    g = synth.erdos_renyi(nv, 0.2, 3, wmax=10)
    if sizes == "uneven":
        sizes = synth.uneven_sizes(nv, 12, 24, 1)
        M = len(sizes)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, M, mode, sizes)
    try:
        first, size, edges, weight = capi.paraqaoa_part_info(part)
        of, osz = orc.partition(nv, M, mode, sizes)
        assert np.array_equal(first, of) and np.array_equal(size, osz)
        for i in range(M):
            s = orc.get_subgraph(g, int(of[i]), int(osz[i]))
            u, v, w = capi.paraqaoa_part_edges(part, i, int(edges[i]))
            assert np.array_equal(u, s.eu) and np.array_equal(v, s.ev) and np.array_equal(w, s.ew)
            assert weight[i] == s.total_weight
    finally:
        capi.paraqaoa_part_free(part)


def test_partition_rejects_bad_input(capi):
    g = synth.erdos_renyi(30, 0.3, 1)
    G = capi.Graph.of(g)
    with pytest.raises(capi.ParaQAOAError) as e:
        capi.paraqaoa_partition(G, 0)
    assert e.value.code == capi.E_INVAL
    with pytest.raises(capi.ParaQAOAError):
        capi.paraqaoa_partition(G, 3, capi.PART_SIZES, [10, 10, 10])  # covers 28, not 30
    with pytest.raises(capi.ParaQAOAError):
        capi.paraqaoa_partition(G, 3, 7)
    # an asymmetric CSR is refused
    bad = capi.Graph(3, [0, 1, 1, 1], [1], [1])
    with pytest.raises(capi.ParaQAOAError):
        capi.paraqaoa_partition(bad, 1)
    # a self-loop is refused
    loop = capi.Graph(2, [0, 1, 1], [0], [1])
    with pytest.raises(capi.ParaQAOAError):
        capi.paraqaoa_partition(loop, 1)


def test_create_fails_loudly_without_gpu(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(capi.ParaQAOAError) as e:
        capi.paraqaoa_create(0)
    assert e.value.code in (capi.E_CUDA, capi.E_INVAL)



def test_pei_efficiency_factor(capi):
    """Sec. 3.5: EF = 0.5 at T_ALG = T_Base (the paper's worked fact, stored
    in tests/golden/paper_examples.json), EF -> 1 when the run is far faster
    than the baseline and -> 0 when far slower, and PEI = AR x EF x 100."""
    import json
    import math
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))
    ef, pei = capi.paraqaoa_pei(0.9, 12.0, 12.0, 1e-3)
    assert ef == gold["efficiency_factor"]["ef_at_parity"] and pei == pytest.approx(45.0)
    ef_fast, _ = capi.paraqaoa_pei(1.0, 0.0, 1e5, 1e-3)
    ef_slow, _ = capi.paraqaoa_pei(1.0, 1e5, 0.0, 1e-3)
    assert ef_fast > 1 - 1e-12 and ef_slow < 1e-12
    # alpha 0.001 per second: a run 1000 s faster than the baseline gets 1 / (1 + e^-1)
    ef, pei = capi.paraqaoa_pei(0.8, 0.0, 1000.0, 1e-3)
    assert ef == pytest.approx(1 / (1 + math.exp(-1))) and pei == pytest.approx(80 * ef)
    with pytest.raises(capi.ParaQAOAError):
        capi.paraqaoa_pei(0.9, -1.0, 1.0, 1e-3)


def test_probe_streams_validates_arguments(capi):
    """The HBM stream probe rejects buffer sizes outside 1 MiB .. 16 GiB or not
    a multiple of 16 bytes before it touches a device."""
    for nbytes in (0, (1 << 20) - 16, (1 << 34) + 16, (1 << 24) + 8, -(1 << 24)):
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_probe_streams(0, nbytes)
        assert e.value.code == capi.E_INVAL
