"""te_evolve (the whole restart cycle on the GPU) against the oracle.

Parity bar: ||v_gpu - v_oracle||_2 <= 2 tol + 1e-12 (both are within tol of the
exact exp(-iHt)v, eq. errorIntegral), on the same seeded inputs.  Step
sequences may differ (sin/cos rounding can flip an accept/reject), so they
are not compared.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse

import workloads as W
from oracle import krylov, models, dense
from oracle.krylov import Options

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


def gpu_evolve(te, ctx, H, v0, t, tol, m, device=True, allow=None, **opt):
    import torch
    o = te.make_options(**opt)
    vin = torch.from_numpy(v0).cuda() if device else v0
    kw = {} if allow is None else {"allow": allow}
    out, st, s = te.te_evolve(ctx, H, vin, t, tol, m, o, **kw)
    return (out.cpu().numpy() if device else out), st, s


def parity(te, ctx, params_or_csr, v0, t, tol, m, oopt=None, **gopt):
    if isinstance(params_or_csr, dict):
        H = te.te_build_model(ctx, params_or_csr)
        A = models.build(params_or_csr).to_scipy()
    else:
        A = params_or_csr.to_scipy()
        c = A.tocoo()
        H = te.te_build_csr(ctx, A.shape[0], c.row, c.col, c.data)
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, v0, t, tol, m, **gopt)
        ref = krylov.evolve(A, v0, t, tol, m, oopt or Options())
        diff = np.linalg.norm(vg - ref.v)
        assert diff <= 2 * tol + 1e-12, (diff, st, ref.restarts)
        assert st["err_bound"] <= tol * (1 + 1e-12)
        assert st["t_reached"] == t
        assert st["m_used"] == min(m, A.shape[0])
        return vg, st, ref, A
    finally:
        te.te_matrix_free(H)


def test_tfim_L12_workload(te, ctx):
    """TFIM L = 12 (d = 4096), t = 10, m = 40, tol = 1e-8; also against the dense definition."""
    wl = W.workload("tfim_L12")
    v0 = W.initial_vector(wl["v0"], wl["d"])
    vg, st, ref, A = parity(te, ctx, wl["params"], v0, wl["t"], wl["tol"], wl["m"])
    exact = dense.expm_apply(A, v0, wl["t"])
    assert np.linalg.norm(vg - exact) <= st["err_bound"] + 1e-12
    assert st["matvecs"] == ref.matvecs or abs(st["restarts"] - ref.restarts) <= 2


@pytest.mark.parametrize("L,t,tol,m", [(10, 7.0, 1e-8, 30), (12, -5.0, 1e-10, 40), (9, 20.0, 1e-6, 12)])
def test_xxzdm(te, ctx, L, t, tol, m):
    p = W.xxzdm_params(L, seed=40 + L)
    v0 = W.random_state(41 + L, 1 << L)
    parity(te, ctx, p, v0, t, tol, m)


def test_bose_small(te, ctx):
    p = W.bose_params(8, 5, seed=44)
    b = models.BoseBasis(8, 5)
    v0 = W.basis_state(len(b), b.index[(1, 1, 1, 1, 1, 0, 0, 0)])
    parity(te, ctx, p, v0, 5.0, 1e-10, 50)


def test_random_hermitian_ragged(te, ctx):
    d = 700
    u = W.uniform(45, 5 * d)
    lens = np.floor(40 * u[:d] ** 3).astype(np.int64)
    rows = np.repeat(np.arange(d), lens)
    n = rows.size
    v = W.uniform(46, 3 * n)
    cols = (v[:n] * d).astype(np.int64)
    vals = (v[n:2 * n] - 0.5) + 1j * (v[2 * n:] - 0.5)
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(d, d))
    A = (A + A.getH()).tocsr()
    A.sum_duplicates()
    csr = models.CSR(d, A.indptr.astype(np.int64), A.indices.astype(np.int64), A.data)
    parity(te, ctx, csr, W.random_state(47, d), 6.0, 1e-8, 35)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_every_spmv_variant(te, ctx, lanes):
    p = W.xxzdm_params(11, seed=48)
    parity(te, ctx, p, W.random_state(49, 1 << 11), 3.0, 1e-8, 25, spmv_lanes=lanes)


@pytest.mark.parametrize("small_exp", ["cheb", "eig"])
@pytest.mark.parametrize("params,v0seed,t,tol,m", [
    (W.xxzdm_params(10, seed=63), 64, 8.0, 1e-8, 30),
    (W.tfim_params(11, seed=65), 66, -12.0, 1e-10, 40),
    (W.bose_params(7, 4, seed=67), 68, 4.0, 1e-6, 15),
], ids=["xxzdm10", "tfim11", "bose7_4"])
def test_small_exponential_methods(te, ctx, small_exp, params, v0seed, t, tol, m):
    """Both evaluations of exp(-i H_m tau) e_1 (Chebyshev series, diagonalisation)."""
    d = models.build(params).d
    parity(te, ctx, params, W.random_state(v0seed, d), t, tol, m, small_exp=small_exp)


@pytest.mark.parametrize("quad,reorth", [("gauss", False), ("tanh-sinh", True), ("gauss", True)])
def test_options(te, ctx, quad, reorth):
    p = W.xxzdm_params(10, seed=50)
    parity(te, ctx, p, W.random_state(51, 1 << 10), 6.0, 1e-8, 25,
           oopt=Options(quad=quad, reorth=reorth), quad=quad, reorth=reorth)


def test_host_buffers(te, ctx):
    p = W.tfim_params(9, seed=52)
    parity(te, ctx, p, W.random_state(53, 512), 4.0, 1e-8, 20, device=False)


def test_rabi_breakdown_closed_form(te, ctx):
    D, O = 0.7, 1.3
    A = 0.5 * np.array([[D, O], [O, -D]], dtype=complex)
    H = te.te_build_csr(ctx, 2, [0, 0, 1, 1], [0, 1, 0, 1], A.reshape(-1))
    try:
        v0 = np.array([1.0, 0.0], dtype=complex)
        for t in [0.3, 5.0, 40.0]:
            w = 0.5 * math.hypot(D, O)
            exact = math.cos(w * t) * v0 - 1j * math.sin(w * t) / w * (A @ v0)
            vg, st, _ = gpu_evolve(te, ctx, H, v0, t, 1e-8, 40)
            assert np.linalg.norm(vg - exact) <= 1e-12
            assert st["breakdowns"] == 1 and st["restarts"] == 1 and st["matvecs"] == 2
            assert st["flags"] & te.TE_FLAG_BREAKDOWN
    finally:
        te.te_matrix_free(H)


def test_decoupled_spins_closed_form(te, ctx):
    L = 12
    p = W.tfim_params(L, seed=54)
    p["J"] = np.zeros(L - 1)
    H = te.te_build_model(ctx, p)
    try:
        t = 3.0
        vg, st, _ = gpu_evolve(te, ctx, H, W.basis_state(1 << L, 0), t, 1e-9, 30)
        r = np.arange(1 << L)
        exact = np.ones(1 << L, dtype=complex)
        for i in range(L):
            exact *= np.where(((r >> i) & 1) == 0, math.cos(p["h"][i] * t), 1j * math.sin(p["h"][i] * t))
        assert np.linalg.norm(vg - exact) <= st["err_bound"] + 1e-12
    finally:
        te.te_matrix_free(H)


def test_one_site_and_t_zero(te, ctx):
    H = te.te_build_csr(ctx, 1, [0], [0], [1.7])
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, np.array([1j]), 2.0, 1e-8, 10)
        assert abs(vg[0] - 1j * np.exp(-1j * 1.7 * 2.0)) < 1e-14
    finally:
        te.te_matrix_free(H)
    p = W.tfim_params(6, seed=55)
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(56, 64)
        vg, st, _ = gpu_evolve(te, ctx, H, v0, 0.0, 1e-8, 10)
        assert np.array_equal(vg, v0) and st["restarts"] == 0
    finally:
        te.te_matrix_free(H)


def test_errors_match_oracle(te, ctx):
    p = W.tfim_params(8, seed=57)
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(58, 256)
        # m = 1: constant integrand h, the step underflows on both sides
        vg, st, s = gpu_evolve(te, ctx, H, v0, 1.0, 1e-8, 1, allow=(te.TE_ERR_STEP_UNDERFLOW,))
        assert s == te.TE_ERR_STEP_UNDERFLOW
        assert krylov.evolve(models.build(p).to_scipy(), v0, 1.0, 1e-8, 1).status == "step_underflow"
        assert np.array_equal(vg, v0)            # state at the time reached (0)
        with pytest.raises(te.TEError) as e:
            gpu_evolve(te, ctx, H, 1.01 * v0, 1.0, 1e-8, 10)
        assert e.value.status == te.TE_ERR_NOT_NORMALIZED
        bad = v0.copy()
        bad[3] = np.nan
        with pytest.raises(te.TEError) as e:
            gpu_evolve(te, ctx, H, bad, 1.0, 1e-8, 10)
        assert e.value.status == te.TE_ERR_NONFINITE
        with pytest.raises(te.TEError) as e:
            gpu_evolve(te, ctx, H, v0, 1.0, 0.0, 10)
        assert e.value.status == te.TE_ERR_INVALID_ARG
        with pytest.raises(te.TEError) as e:
            gpu_evolve(te, ctx, H, v0, 1.0, 1e-8, te.TE_M_MAX + 1)
        assert e.value.status == te.TE_ERR_UNSUPPORTED
    finally:
        te.te_matrix_free(H)


def test_m_max_and_roundoff_warning(te, ctx):
    p = W.xxzdm_params(12, seed=59)
    v0 = W.random_state(60, 1 << 12)
    vg, st, ref, A = parity(te, ctx, p, v0, 30.0, 1e-12, te.TE_M_MAX)
    assert bool(st["flags"] & te.TE_WARN_ROUNDOFF) == ref.warn_roundoff
    per_gpu = st["roundoff_est"] / st["restarts"]
    per_ref = ref.roundoff_est / ref.restarts
    assert abs(per_gpu - per_ref) <= 1e-12 * per_ref


def test_profile_counts_spmv_launches(te, ctx):
    p = W.tfim_params(10, seed=61)
    H = te.te_build_model(ctx, p)
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, W.random_state(62, 1024), 5.0, 1e-8, 30, profile=True)
        # one timed product (Lanczos step m/2) per restart that reached it
        assert 0 < st["spmv_launches"] <= st["restarts"] and st["spmv_ms"] > 0
        assert st["spmv_launches"] == st["restarts"] - st["breakdowns"]
    finally:
        te.te_matrix_free(H)


# ---------------------------------------------------------------- full workload sizes

def test_xxzdm_L22_one_restart_against_oracle(te, ctx):
    """Full-size XXZ-DM (d = 4,194,304): a time short enough for a single
    restart, compared with the oracle element by element."""
    wl = W.workload("xxzdm_L22")
    p = wl["params"]
    v0 = W.initial_vector(wl["v0"], wl["d"])
    H = te.te_build_model(ctx, p)
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, v0, 0.4, wl["tol"], wl["m"])
    finally:
        te.te_matrix_free(H)
    ref = krylov.evolve(models.xxzdm_csr(p).to_scipy(), v0, 0.4, wl["tol"], wl["m"])
    assert ref.restarts == 1
    assert np.linalg.norm(vg - ref.v) <= 2 * wl["tol"] + 1e-12


def test_xxzdm_L22_several_restarts_against_oracle(te, ctx):
    """Full-size XXZ-DM (d = 4,194,304) over t = 5 (several restarts, with the
    shrink and growth of the step search between them), element by element
    against the oracle (its product on all host cores)."""
    wl = W.workload("xxzdm_L22")
    p = wl["params"]
    v0 = W.initial_vector(wl["v0"], wl["d"])
    H = te.te_build_model(ctx, p)
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, v0, 5.0, wl["tol"], wl["m"])
    finally:
        te.te_matrix_free(H)
    ref = krylov.evolve(models.xxzdm_csr(p).to_scipy(), v0, 5.0, wl["tol"], wl["m"],
                        threads=os.cpu_count())
    assert ref.restarts >= 3 and st["restarts"] >= 3
    assert np.linalg.norm(vg - ref.v) <= 2 * wl["tol"] + 1e-12


def test_bose_K14_N10_restarts_against_oracle(te, ctx):
    """Full-size bosonic workload (d = 1,144,066, rows of 14..131 entries, the
    value-indexed copy with ~4,900 distinct couplings), tol = 1e-10, m = 50, over
    a time of two to three restarts, element by element against the oracle."""
    wl = W.workload("bose_K14_N10")
    p = wl["params"]
    b = models.BoseBasis(14, 10)
    v0 = W.basis_state(wl["d"], b.index[wl["v0"][1]])
    H = te.te_build_model(ctx, p)
    try:
        vg, st, _ = gpu_evolve(te, ctx, H, v0, 0.6, wl["tol"], wl["m"])
    finally:
        te.te_matrix_free(H)
    A = models.bose_csr_vec(p, b).to_scipy()
    ref = krylov.evolve(A, v0, 0.6, wl["tol"], wl["m"], threads=os.cpu_count())
    assert ref.restarts >= 2 and st["restarts"] >= 2
    assert np.linalg.norm(vg - ref.v) <= 2 * wl["tol"] + 1e-12


def test_xxzdm_L22_full_solve_properties(te, ctx):
    """The bench workload (t = 50, m = 40, tol = 1e-8) in the bench's launch
    configuration: the reported bound, the final time, norm and S^z sector
    (components outside the Neel sector stay exactly 0), and the forward-backward
    return of Sec. 5 within 2 tol."""
    import torch
    wl = W.workload("xxzdm_L22")
    d, t, tol, m = wl["d"], wl["t"], wl["tol"], wl["m"]
    v0 = W.initial_vector(wl["v0"], d)
    H = te.te_build_model(ctx, wl["params"])
    try:
        o = te.make_options()
        fwd, st, _ = te.te_evolve(ctx, H, torch.from_numpy(v0).cuda(), t, tol, m, o)
        assert st["err_bound"] <= tol and st["t_reached"] == t
        assert abs(torch.linalg.vector_norm(fwd).item() - 1.0) <= tol
        r = torch.arange(d, device="cuda")
        pop = torch.zeros(d, dtype=torch.int64, device="cuda")
        for i in range(22):
            pop += (r >> i) & 1
        assert torch.count_nonzero(fwd[pop != 11]).item() == 0
        back, st2, _ = te.te_evolve(ctx, H, fwd, -t, tol, m, o)
        err = torch.linalg.vector_norm(back.cpu() - torch.from_numpy(v0)).item()
        assert err <= 2 * tol + 1e-12
    finally:
        te.te_matrix_free(H)


def test_bose_K14_N10_forward_backward(te, ctx):
    """Full-size bosonic workload (ragged rows 14..131): forward-backward within
    2 tol plus the roundoff estimate, which exceeds tol here (Sec. 5 reports the
    same warning for its d = 1.5e6 example)."""
    import torch
    wl = W.workload("bose_K14_N10")
    p = wl["params"]
    idx = te.te_model_basis_index(p, wl["v0"][1])
    d = wl["d"]
    v0 = W.basis_state(d, idx)
    H = te.te_build_model(ctx, p)
    try:
        o = te.make_options()
        t, tol, m = 2.0, wl["tol"], wl["m"]
        fwd, st, _ = te.te_evolve(ctx, H, torch.from_numpy(v0).cuda(), t, tol, m, o)
        assert st["err_bound"] <= tol
        back, _, _ = te.te_evolve(ctx, H, fwd, -t, tol, m, o)
        err = torch.linalg.vector_norm(back.cpu() - torch.from_numpy(v0)).item()
        assert err <= 2 * tol + 1e-12 + st["roundoff_est"]
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("L,t", [(12, 6.0), (20, 0.5)])
def test_general_complex_csr_full_value_form(te, ctx, L, t):
    """A general complex Hermitian matrix from COO with a distinct value per coupled
    pair (more than the value table's 65,535 at L = 20): the full-value sliced copy
    is the product, and the solve equals the oracle's within 2 tol + 1e-12."""
    rows, cols, vals = W.random_hermitian_coo(L, 9)
    d = 1 << L
    H = te.te_build_csr(ctx, d, rows, cols, vals)
    try:
        info = te.te_matrix_info_get(H)
        if L == 20:
            assert info["sell_dict"] == 0                # full-value form
        v0 = W.random_state(309, d)
        vg, st, _ = gpu_evolve(te, ctx, H, v0, t, 1e-8, 40)
    finally:
        te.te_matrix_free(H)
    A = models.coo_to_csr(d, rows, cols, vals).to_scipy()
    ref = krylov.evolve(A, v0, t, 1e-8, 40, threads=os.cpu_count())
    assert np.linalg.norm(vg - ref.v) <= 2e-8 + 1e-12
    assert st["t_reached"] == t and st["err_bound"] <= 1e-8
