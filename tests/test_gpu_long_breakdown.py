"""Lucky breakdowns that take a long remaining time in one step (Sec. 2.4 step 1,
eq. krylovApproximation), on every engine, against the oracle.

After a breakdown the whole remaining time t_rem is one step, so
exp(-i H_m t_rem) e_1 is needed at an argument ||H_m|| t_rem that the step
search never reaches.  The library's Chebyshev/Bessel evaluation splits such a
step into pieces; these tests check it element by element against the oracle
(which diagonalises H_m and has no range limit) and against closed forms:

* an eigenvector input (diagonal H, basis state): m_eff = 1, v(t) = e^{-i E t} v;
* the 14-mode, one-boson model (d = 14 < m): H is the 14 x 14 coupling matrix;
  at tol = 1e-6 the 14th Lanczos step breaks down (h_{15,14} ~ 1e-11 < tol / t),
  at tol = 1e-8 it does not and the step search alone covers t;
* the two-level Rabi problem far beyond one series piece.

Parity bar: ||v_gpu - v_oracle||_2 <= 2 tol + 1e-12.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense, krylov, models

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


@pytest.fixture(scope="module")
def diag_matrix(te, ctx):
    d = 16
    e = 2.0 * W.uniform(910, d) - 1.0
    H = te.te_build_csr(ctx, d, np.arange(d), np.arange(d), e.astype(complex))
    yield H, e
    te.te_matrix_free(H)


@pytest.fixture(scope="module")
def one_boson(te, ctx):
    p = W.bose_params(14, 1, seed=911)
    H = te.te_build_model(ctx, p)
    yield H, models.build(p).to_scipy()
    te.te_matrix_free(H)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("small_exp", ["cheb", "eig"])
@pytest.mark.parametrize("t", [5000.0, -5000.0])
def test_eigenvector_input_long_time(te, ctx, diag_matrix, small_exp, t):
    """m_eff = 1: the step is exp(-i alpha_1 t) applied to v (closed form)."""
    H, e = diag_matrix
    k = 5
    v0 = W.basis_state(e.size, k)
    out, st, _ = te.te_evolve(ctx, H, _dev(v0), t, TOL, 40, te.make_options(small_exp=small_exp))
    vg = out.cpu().numpy()
    ref = krylov.evolve(np.diag(e.astype(complex)), v0, t, TOL, 40)
    assert np.linalg.norm(vg - ref.v) <= 2 * TOL + 1e-12
    exact = np.exp(-1j * e[k] * t) * v0
    # the phase e_k t is rounded once on each side: |t| e_k 2^-52 of difference
    assert np.linalg.norm(vg - exact) <= 4 * abs(t) * 2.0 ** -52 + 1e-14
    assert st["breakdowns"] == 1 and st["restarts"] == 1 and st["t_reached"] == t


@pytest.mark.parametrize("small_exp", ["cheb", "eig"])
@pytest.mark.parametrize("tol", [1e-8, 1e-6])
@pytest.mark.parametrize("t", [1000.0, -1000.0])
def test_one_boson_long_time(te, ctx, one_boson, small_exp, tol, t):
    """d = 14 < m = 40: the Krylov space is the whole space."""
    H, A = one_boson
    v0 = W.random_state(912, 14)
    out, st, _ = te.te_evolve(ctx, H, _dev(v0), t, tol, 40, te.make_options(small_exp=small_exp))
    vg = out.cpu().numpy()
    ref = krylov.evolve(A, v0, t, tol, 40)
    assert np.linalg.norm(vg - ref.v) <= 2 * tol + 1e-12
    assert np.linalg.norm(vg - dense.expm_apply(A, v0, t)) <= st["err_bound"] + 1e-10
    assert st["t_reached"] == t and st["m_used"] == 14
    if tol == 1e-6:
        assert st["breakdowns"] == 1 and st["restarts"] == 1


def test_rabi_far_beyond_one_piece(te, ctx):
    """d = 2, Omega t up to 2e5 (about 100 series pieces): the closed form
    cos(w t) v - i sin(w t)/w H v, within the phase rounding |t| ||H|| 2^-52."""
    D, O = 0.7, 1.3
    A = 0.5 * np.array([[D, O], [O, -D]], dtype=complex)
    H = te.te_build_csr(ctx, 2, [0, 0, 1, 1], [0, 1, 0, 1], A.reshape(-1))
    try:
        v0 = np.array([1.0, 0.0], dtype=complex)
        w = 0.5 * math.hypot(D, O)
        for t in (3.0e3, 1.0e4, 2.0e5):
            exact = math.cos(w * t) * v0 - 1j * math.sin(w * t) / w * (A @ v0)
            out, st, _ = te.te_evolve(ctx, H, _dev(v0), t, TOL, 40)
            vg = out.cpu().numpy()
            assert np.linalg.norm(vg - exact) <= 64 * t * 2.0 ** -52 + 1e-12, t
            ref = krylov.evolve(A, v0, t, TOL, 40)
            assert np.linalg.norm(vg - ref.v) <= 2 * TOL + 1e-12, t
            assert st["breakdowns"] == 1 and st["restarts"] == 1
    finally:
        te.te_matrix_free(H)


def test_beyond_the_piece_limit_is_an_error_not_a_wrong_answer(te, ctx):
    """||H_m|| t above 2048 x 512: the series reports TE_ERR_UNSUPPORTED; the
    diagonalisation option evaluates the same step."""
    D, O = 0.7, 1.3
    A = 0.5 * np.array([[D, O], [O, -D]], dtype=complex)
    H = te.te_build_csr(ctx, 2, [0, 0, 1, 1], [0, 1, 0, 1], A.reshape(-1))
    try:
        v0 = np.array([1.0, 0.0], dtype=complex)
        t = 2.0e6
        _, _, s = te.te_evolve(ctx, H, _dev(v0), t, TOL, 40, allow=(te.TE_ERR_UNSUPPORTED,))
        assert s == te.TE_ERR_UNSUPPORTED
        assert "series" in te.te_last_error(ctx)
        out, st, _ = te.te_evolve(ctx, H, _dev(v0), t, TOL, 40, te.make_options(small_exp="eig"))
        w = 0.5 * math.hypot(D, O)
        exact = math.cos(w * t) * v0 - 1j * math.sin(w * t) / w * (A @ v0)
        assert np.linalg.norm(out.cpu().numpy() - exact) <= 64 * t * 2.0 ** -52
        # the context still solves afterwards
        out, st, _ = te.te_evolve(ctx, H, _dev(v0), 1.0, TOL, 40)
        assert st["t_reached"] == 1.0
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("small_exp", ["cheb", "eig"])
def test_batch_long_breakdown(te, ctx, one_boson, small_exp):
    """te_evolve_batch: several vectors under the d = 14 Hamiltonian at t = 1000."""
    H, A = one_boson
    nvec = 5
    V0 = np.stack([W.random_state(913 + b, 14) for b in range(nvec)])
    t, tol = 1000.0, 1e-6
    out, sts, stat, _ = te.te_evolve_batch(ctx, H, _dev(V0), t, tol, 40,
                                           te.make_options(small_exp=small_exp))
    out = out.cpu().numpy()
    for b in range(nvec):
        assert stat[b] == te.TE_OK
        ref = krylov.evolve(A, V0[b], t, tol, 40)
        assert np.linalg.norm(out[b] - ref.v) <= 2 * tol + 1e-12, b
        assert sts[b]["t_reached"] == t and sts[b]["breakdowns"] == 1


@pytest.mark.parametrize("small_exp", ["cheb", "eig"])
def test_multi_long_breakdown(te, ctx, diag_matrix, one_boson, small_exp):
    """te_evolve_multi: the eigenvector problem (t = 5000), the one-boson problem
    (t = 1000) and an ordinary spin chain, advanced together."""
    Hd, e = diag_matrix
    Hb, A = one_boson
    p = W.xxzdm_params(9, seed=914)
    Hx = te.te_build_model(ctx, p)
    try:
        Ax = models.build(p).to_scipy()
        vs = [W.basis_state(e.size, 3), W.random_state(915, 14), W.random_state(916, Ax.shape[0])]
        ts = [5000.0, -1000.0, 6.0]
        tol = 1e-6
        mats = [np.diag(e.astype(complex)), A, Ax]
        outs, sts, stat, _ = te.te_evolve_multi(ctx, [Hd, Hb, Hx], [_dev(v) for v in vs], ts, tol,
                                                30, te.make_options(small_exp=small_exp))
        for i in range(3):
            assert stat[i] == te.TE_OK, i
            ref = krylov.evolve(mats[i], vs[i], ts[i], tol, 30)
            assert np.linalg.norm(outs[i].cpu().numpy() - ref.v) <= 2 * tol + 1e-12, i
            assert sts[i]["t_reached"] == ts[i]
        assert sts[0]["breakdowns"] == 1 and sts[1]["breakdowns"] == 1
    finally:
        te.te_matrix_free(Hx)


@pytest.mark.parametrize("tol", [1e-8, 1e-6])
def test_sampled_long_breakdown(te, ctx, one_boson, tol):
    """te_evolve_sampled: samples inside the single long step after the breakdown."""
    H, A = one_boson
    v0 = W.random_state(916, 14)
    t = 1000.0
    ts = [0.0, 1.5, 333.3, 999.0, 1000.0]
    out, samp, _, bounds, st, _ = te.te_evolve_sampled(ctx, H, _dev(v0), t, ts, tol, 40)
    samp = samp.cpu().numpy()
    ref = krylov.evolve(A, v0, t, tol, 40, samples=ts)
    for k, s in enumerate(ts):
        assert np.linalg.norm(samp[k] - ref.samples[k]) <= 2 * tol + 1e-12, k
        assert np.linalg.norm(samp[k] - dense.expm_apply(A, v0, s)) <= bounds[k] + 1e-10, k
    assert np.linalg.norm(out.cpu().numpy() - ref.v) <= 2 * tol + 1e-12
