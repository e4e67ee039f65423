"""The allocation-free top-K entry point against the context-owned one.

paraqaoa_topk_noalloc serves callers that must not let a library allocate
device memory (a host whose own allocator already holds the device memory,
or a latency-critical loop that cannot take cudaMalloc's synchronisation).
Called through the C ABI on device buffers, it must return what
paraqaoa_topk returns for the same states; the calls run back to back, so
one call's leftovers in the shared scratch array would show up in the next.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_topk_matches_context_topk():
    import torch

    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi as capi

    ctx = capi.paraqaoa_create(0)
    try:
        sizes = [12, 17, 20]
        g = synth.erdos_renyi(int(sum(sizes)) - 2, 0.4, 9, wmax=10)
        part = capi.paraqaoa_partition(capi.Graph.of(g), 3, capi.PART_SIZES, sizes)
        try:
            ids = np.arange(3, dtype=np.int32)
            gam, bet = synth.random_angles(3, 2, 11)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_KEEP_STATE)
            states = [capi.paraqaoa_state(ctx, i, n) for i, n in enumerate(sizes)]
            stream = torch.cuda.current_stream()
            for K, flags in [(16, capi.TOPK_CANONICAL), (32, capi.TOPK_RAW)]:
                z_ref, p_ref = capi.paraqaoa_topk(ctx, 3, K, flags)
                for i, n in enumerate(sizes):
                    d_state = torch.from_numpy(states[i].view(np.float32).copy()).cuda()
                    for _ in range(2):  # two calls in a row on the shared scratch
                        d_z = torch.full((K,), -1, dtype=torch.int32, device="cuda")
                        d_p = torch.full((K,), -1.0, dtype=torch.float32, device="cuda")
                        capi.paraqaoa_topk_noalloc(d_state.data_ptr(), n, K, d_z.data_ptr(), d_p.data_ptr(),
                                                   flags, stream.cuda_stream)
                        stream.synchronize()
                        z = d_z.cpu().numpy().view(np.uint32)
                        pr = d_p.cpu().numpy()
                        assert np.array_equal(z, z_ref[i]), (n, K, flags)
                        assert np.max(np.abs(pr - p_ref[i])) <= 1e-5 * float(p_ref[i].max())
        finally:
            capi.paraqaoa_part_free(part)
    finally:
        capi.paraqaoa_destroy(ctx)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    import torch

    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi as capi

    dummy = torch.zeros(64, dtype=torch.float32, device="cuda")
    out_z = torch.zeros(4, dtype=torch.int32, device="cuda")
    out_p = torch.zeros(4, dtype=torch.float32, device="cuda")
    # 2^26 canonical entries (n = 27) or 2^26 raw entries (n = 26) exceed the 2^25 limit;
    # the call refuses before touching the buffers
    for n, flags in [(27, capi.TOPK_CANONICAL), (26, capi.TOPK_RAW)]:
        with pytest.raises(capi.ParaQAOAError) as e:
            capi.paraqaoa_topk_noalloc(dummy.data_ptr(), n, 4, out_z.data_ptr(), out_p.data_ptr(), flags, None)
        assert e.value.code == capi.E_SCRATCH_LIMIT


def test_noalloc_topk_at_the_scratch_limit():
    """n = 25 ranked raw is exactly 2^25 entries: every chunk of the fixed
    scratch array is used. Two calls in a row must both equal the
    context-owned paraqaoa_topk of the same 256 MB state."""
    import torch

    import paper_2603_26232_gb300 as pkg
    pkg.build()
    from paper_2603_26232_gb300 import _capi as capi

    ctx = capi.paraqaoa_create(0)
    try:
        n, K = 25, 32
        g = synth.erdos_renyi(n, 0.3, 25, wmax=10)
        part = capi.paraqaoa_partition(capi.Graph.of(g), 1)
        try:
            ids = np.zeros(1, np.int32)
            gam, bet = synth.random_angles(1, 2, 25)
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_KEEP_STATE)
            z_ref, p_ref = capi.paraqaoa_topk(ctx, 1, K, capi.TOPK_RAW)
            d_state = torch.from_numpy(capi.paraqaoa_state(ctx, 0, n).view(np.float32)).cuda()
            stream = torch.cuda.current_stream()
            for _ in range(2):
                d_z = torch.full((K,), -1, dtype=torch.int32, device="cuda")
                d_p = torch.full((K,), -1.0, dtype=torch.float32, device="cuda")
                capi.paraqaoa_topk_noalloc(d_state.data_ptr(), n, K, d_z.data_ptr(), d_p.data_ptr(),
                                           capi.TOPK_RAW, stream.cuda_stream)
                stream.synchronize()
                assert np.array_equal(d_z.cpu().numpy().view(np.uint32), z_ref[0])
                assert np.max(np.abs(d_p.cpu().numpy() - p_ref[0])) <= 1e-5 * float(p_ref[0].max())
            del d_state
        finally:
            capi.paraqaoa_part_free(part)
    finally:
        capi.paraqaoa_destroy(ctx)
