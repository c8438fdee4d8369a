"""te_create_with_allocator: every device buffer of the library from a caller's
allocator (here PyTorch's caching allocator through ctypes callbacks).

The TFIM L = 12 workload (d = 4096, t = 10, m = 40, tol = 1e-8) is solved on a
context whose allocator is torch's pool: the result equals the oracle within
2 tol + 1e-12 and the default context's result bit for bit, torch's
memory_allocated covers the library's workspace (the (m+1) d complex128 Krylov
basis among it), and everything goes back to the pool when the matrix and the
context are released.  A request (te_submit) takes its buffers from the same
allocator on the scheduler's worker thread.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov, models

pytestmark = pytest.mark.gpu


def test_torch_caching_allocator_holds_the_workspace(te):
    import torch
    torch.cuda.set_device(0)
    wl = W.workload("tfim_L12")
    d, t, tol, m = wl["d"], wl["t"], wl["tol"], wl["m"]
    v0 = W.initial_vector(wl["v0"], d)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(0)
    alloc = te.TorchAllocator()
    ctx = te.te_create(0, allocator=alloc)
    try:
        assert alloc.bytes_live() > 0                      # the context's own scratch
        H = te.te_build_model(ctx, wl["params"])
        try:
            vin = torch.from_numpy(v0).cuda()
            out, st, _ = te.te_evolve(ctx, H, vin, t, tol, m)
            torch.cuda.synchronize()
            live = alloc.bytes_live()
            basis = (m + 1) * d * 16
            assert live >= basis + 20 * 53248               # Krylov basis and the CSR arrays
            # vin and out are torch's own tensors; the rest is the library's
            assert torch.cuda.memory_allocated(0) - base >= live + 2 * d * 16
            ref = krylov.evolve(models.build(wl["params"]).to_scipy(), v0, t, tol, m)
            assert np.linalg.norm(out.cpu().numpy() - ref.v) <= 2 * tol + 1e-12
            # the same solve on a cudaMalloc context: bitwise the same state
            c2 = te.te_create(0)
            try:
                H2 = te.te_build_model(c2, wl["params"])
                out2, _, _ = te.te_evolve(c2, H2, vin, t, tol, m)
                te.te_matrix_free(H2)
                assert torch.equal(out, out2)
                del out2
            finally:
                te.te_destroy(c2)
            # a request: its buffers come from the allocator on a worker thread
            req = te.te_submit(ctx, H, v0, t, tol, m)
            vreq = np.empty(d, dtype=np.complex128)
            s, _ = te.te_wait(req, 120000.0, v_out=vreq)
            assert s == te.TE_OK
            # served through the grouped kernels: the same steps, other summation order
            assert np.linalg.norm(vreq - out.cpu().numpy()) <= 2 * tol + 1e-12
            te.te_request_free(req)
        finally:
            te.te_matrix_free(H)
        assert alloc.bytes_live() > 0                      # only the context's scratch is left
    finally:
        te.te_destroy(ctx)
    assert alloc.bytes_live() == 0
    torch.cuda.synchronize()
    del vin, out
    assert torch.cuda.memory_allocated(0) == base


def test_allocator_failure_is_an_oom_status(te):
    """An allocator that refuses the large Krylov basis: the solve reports
    TE_ERR_OOM and the context keeps working once memory is available again."""
    import torch
    alloc = te.TorchAllocator()
    real = alloc._afn
    state = {"cap": None}

    def limited(user, nbytes, device, stream):
        if state["cap"] is not None and nbytes > state["cap"]:
            return None
        return real(user, nbytes, device, stream)

    alloc._afn2 = te.TE_ALLOC_FN(limited)
    alloc.struct = te.te_allocator(alloc._afn2, alloc._ffn, None)
    ctx = te.te_create(0, allocator=alloc)
    try:
        p = W.xxzdm_params(12, seed=5)
        H = te.te_build_model(ctx, p)
        try:
            v0 = torch.from_numpy(W.random_state(6, 1 << 12)).cuda()
            state["cap"] = 1 << 16                           # below the (m+1) d basis
            _, _, s = te.te_evolve(ctx, H, v0, 1.0, 1e-8, 30, allow=(te.TE_ERR_OOM,))
            assert s == te.TE_ERR_OOM
            state["cap"] = None
            out, st, s = te.te_evolve(ctx, H, v0, 1.0, 1e-8, 30)
            assert s == te.TE_OK and st["t_reached"] == 1.0
        finally:
            te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)
    assert alloc.bytes_live() == 0


def test_allocator_arguments_are_checked(te):
    import ctypes as C
    half = te.te_allocator(te.TE_ALLOC_FN(lambda *a: None), te.TE_FREE_FN(), None)
    out = C.c_void_p()
    s = te.lib().te_create_with_allocator(C.byref(out), 0, None, C.byref(half))
    assert s == te.TE_ERR_INVALID_ARG
