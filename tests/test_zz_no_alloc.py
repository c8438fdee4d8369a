"""te_spmv_noalloc, the allocation-free SpMV entry point, against the oracle's
A @ x and against te_spmv.

It serves callers that cannot allocate device memory when they need a product
(under a framework that owns all device memory through its own pool, in a
service whose device footprint is fixed once started, or in loops that cannot
pay for cudaMalloc/cudaFree).  Its scratch is a fixed device array shared by
all calls, so the test calls it twice in a row, on different inputs and then on
the same input again, and compares each result element by element with the
oracle's product at the SpMV parity tolerance 1e-14 (|A| |x|)_i, and with the
allocating te_spmv on the same inputs.  After its first (set-up) call it must
not change the device's free memory.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from oracle import models

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_te_spmv_twice(te):
    import torch
    ctx = te.te_create(0)
    try:
        for params in (W.xxzdm_params(14, 91), W.bose_params(10, 5, 92)):
            H = te.te_build_model(ctx, params)
            try:
                d = te.te_matrix_info_get(H)["d"]
                A = models.build(params).to_scipy()
                absA = abs(A)
                for seed in (93, 94, 94):          # two calls in a row on new input, then a repeat
                    xh = W.complex_gaussian(seed, d)
                    x = torch.from_numpy(xh).cuda()
                    y = torch.full_like(x, complex(np.nan, np.nan))
                    dot = te.te_spmv_noalloc(ctx, H, x, y)
                    yg = y.cpu().numpy()
                    # the oracle's product, element by element
                    yo = A @ xh
                    scale = absA @ np.abs(xh)
                    assert np.all(np.abs(yg - yo) <= 1e-14 * scale)
                    assert abs(dot - float(np.vdot(xh, yo).real)) <= 1e-12 * float(np.abs(xh) @ scale)
                    # and the allocating entry point on the same input
                    y_ref, dot_ref = te.te_spmv(ctx, H, x)
                    assert np.all(np.abs(yg - y_ref.cpu().numpy()) <= 1e-14 * scale)
                    assert abs(dot - dot_ref) <= 1e-12 * float(np.abs(xh) @ scale)
            finally:
                te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)


def test_noalloc_leaves_free_device_memory_unchanged(te):
    """After the set-up call, repeated calls allocate no device memory: the
    driver's free-memory figure stays the same.  At d = 2^20 a per-call
    allocation of even one vector (16 MB) would show in it."""
    import torch
    ctx = te.te_create(0)
    try:
        params = W.xxzdm_params(20, 95)
        H = te.te_build_model(ctx, params)
        try:
            d = te.te_matrix_info_get(H)["d"]
            x = torch.from_numpy(W.complex_gaussian(96, d)).cuda()
            y = torch.empty_like(x)
            dot0 = te.te_spmv_noalloc(ctx, H, x, y)            # set-up call
            y0 = y.clone()
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            for _ in range(5):
                dot = te.te_spmv_noalloc(ctx, H, x, y)
                assert dot == dot0
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free1 == free0
            assert torch.equal(y, y0)
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
