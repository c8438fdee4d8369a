"""te_spmv_noalloc, the allocation-free SpMV entry point, against te_spmv.

It serves callers that cannot allocate device memory when they need a product
(under a framework that owns all device memory through its own pool, in a
service whose device footprint is fixed once started, or in loops that cannot
pay for cudaMalloc/cudaFree).  Its scratch is a fixed device
array shared by all calls, so the test calls it twice in a row, on different
inputs and then on the same input again, and compares each result with the
allocating te_spmv on the same inputs.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import scipy.sparse

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_te_spmv_twice(te):
    import torch
    ctx = te.te_create(0)
    try:
        for params in (W.xxzdm_params(14, 91), W.bose_params(10, 5, 92)):
            H = te.te_build_model(ctx, params)
            try:
                d = te.te_matrix_info_get(H)["d"]
                rp, col, val = te.te_matrix_export(ctx, H)
                absA = scipy.sparse.csr_matrix((np.abs(val), col, rp), shape=(d, d))
                for seed in (93, 94, 94):          # two calls in a row on new input, then a repeat
                    xh = W.complex_gaussian(seed, d)
                    x = torch.from_numpy(xh).cuda()
                    y_ref, dot_ref = te.te_spmv(ctx, H, x)
                    y = torch.full_like(x, complex(np.nan, np.nan))
                    dot = te.te_spmv_noalloc(ctx, H, x, y)
                    # the SpMV parity tolerance: 1e-14 (|A| |x|)_i per element
                    scale = absA @ np.abs(xh)
                    diff = np.abs(y.cpu().numpy() - y_ref.cpu().numpy())
                    assert np.all(diff <= 1e-14 * scale)
                    assert abs(dot - dot_ref) <= 1e-12 * float(np.abs(xh) @ scale)
            finally:
                te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)


def test_noalloc_rejects_oversize_and_host_buffers(te):
    import torch
    ctx = te.te_create(0)
    try:
        d = te.TE_NOALLOC_MAX_D + 1
        H = te.te_build_csr(ctx, d, [0, d - 1], [0, d - 1], [1.0, 2.0])
        try:
            x = torch.zeros(d, dtype=torch.complex128, device="cuda")
            y = torch.empty_like(x)
            with pytest.raises(te.TEError) as e:
                te.te_spmv_noalloc(ctx, H, x, y)
            assert e.value.status == te.TE_ERR_UNSUPPORTED
        finally:
            te.te_matrix_free(H)
        H = te.te_build_csr(ctx, 2, [0, 1], [0, 1], [1.0, 2.0])
        try:
            with pytest.raises(te.TEError) as e:
                te.te_spmv_noalloc(ctx, H, np.ones(2, complex), np.ones(2, complex))
            assert e.value.status == te.TE_ERR_INVALID_ARG
        finally:
            te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)
