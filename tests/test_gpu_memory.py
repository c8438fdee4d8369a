"""The paper's example system (Sec. 5) on the GPU: bit-exact CSR against the oracle,
the printed dimensions, parity, and the forward-backward bound."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import krylov, models

pytestmark = pytest.mark.gpu
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_example_system.json")))


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


@pytest.mark.parametrize("kw", [{}, dict(K=5, Kp=5, N0=30, Nm=3, Nc=30.0), dict(K=1, Kp=2, N0=0, Nm=1)])
def test_csr_bitexact(te, ctx, kw):
    p = W.memory_params(**kw)
    b = models.MemoryBasis(p)
    want = models.memory_csr(p, b)
    H = te.te_build_model(ctx, p)
    try:
        rp, col, val = te.te_matrix_export(ctx, H)
        assert np.array_equal(rp.astype(np.int64), want.rowptr)
        assert np.array_equal(col.astype(np.int64), want.col)
        assert np.array_equal(val.view(np.uint64), want.val.view(np.uint64))
        occ = W.memory_initial_occupation(p)
        assert te.te_model_basis_index(p, occ) == b.index(occ)
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("key", ["benchmark", "memory_limit_point"])
def test_printed_dimensions_and_sampled_rows(te, ctx, key):
    g = GOLDEN[key]
    p = W.memory_params(K=g["K"], Kp=g["Kp"], N0=g["N0"], Nm=g["Nm"], Nc=g["Nc"])
    b = models.MemoryBasis(p)
    H = te.te_build_model(ctx, p)
    try:
        info = te.te_matrix_info_get(H)
        assert info["d"] == g["printed_dimension"]
        rp, col, val = te.te_matrix_export(ctx, H)
        u = W.uniform(900, 150)
        for r in np.unique((u * info["d"]).astype(np.int64)).tolist() + [0, info["d"] - 1]:
            c, v = models.memory_row(p, b, r)
            s, e = rp[r], rp[r + 1]
            assert np.array_equal(col[s:e].astype(np.int64), c)
            assert np.array_equal(val[s:e].view(np.uint64), v.view(np.uint64))
        if key == "benchmark":
            assert abs(info["norm1"] - models.memory_norm1(p, b)) <= 1e-13 * info["norm1"]
    finally:
        te.te_matrix_free(H)


def test_parity_and_forward_backward_default_parameters(te, ctx):
    import torch
    g = GOLDEN["forward_backward"]
    p = W.memory_params()
    b = models.MemoryBasis(p)
    v0 = W.basis_state(len(b), b.index(W.memory_initial_occupation(p)))
    H = te.te_build_model(ctx, p)
    try:
        fwd, st, _ = te.te_evolve(ctx, H, torch.from_numpy(v0).cuda(), g["t"], g["err_max"], 40)
        ref = krylov.evolve(models.memory_csr(p, b).to_scipy(), v0, g["t"], g["err_max"], 40)
        assert np.linalg.norm(fwd.cpu().numpy() - ref.v) <= 2 * g["err_max"] + 1e-12
        back, _, _ = te.te_evolve(ctx, H, fwd, -g["t"], g["err_max"], 40)
        assert np.linalg.norm(back.cpu().numpy() - v0) <= g["printed_requested_bound"]
    finally:
        te.te_matrix_free(H)


def test_benchmark_system_roundoff_estimate(te, ctx):
    """Sec. 5: for the benchmark system (t = 10, m = 40, err_max = 1e-7) the roundoff
    estimate of eq. numericalError is 3.2e-6 and a warning is triggered.  The sum of
    the per-restart estimates reproduces it up to the restart count, which depends
    on step-search details (factor 1.5 allowed)."""
    import torch
    g = GOLDEN["benchmark"]
    p = W.memory_params(K=g["K"], Kp=g["Kp"], N0=g["N0"], Nm=g["Nm"], Nc=g["Nc"])
    H = te.te_build_model(ctx, p)
    try:
        d = te.te_matrix_info_get(H)["d"]
        idx = te.te_model_basis_index(p, W.memory_initial_occupation(p))
        v0 = torch.zeros(d, dtype=torch.complex128, device="cuda")
        v0[idx] = 1.0
        out, st, _ = te.te_evolve(ctx, H, v0, g["t"], g["err_max"], g["m"])
        assert st["err_bound"] <= g["err_max"]
        assert st["flags"] & te.TE_WARN_ROUNDOFF
        ratio = st["roundoff_est"] / g["printed_roundoff_estimate"]
        assert 1 / 1.5 <= ratio <= 1.5, (st["roundoff_est"], st["restarts"])
    finally:
        te.te_matrix_free(H)
