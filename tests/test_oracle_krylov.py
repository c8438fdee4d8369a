"""Pins for the oracle's restarted Krylov solve (Algorithm 1).

Each pin comes from outside the oracle: the dense definition exp(-iHt)v
(eq. vOfT), closed forms, the Galerkin relations of Sec. 2.1, the rigour of
eq. errorIntegral checked against a dense unrestarted Krylov error, the
forward-backward check of Sec. 5, and step-size rules checked on integrals
with a known answer.  A few tests plant a plausible mistake in the oracle and
check that a pin catches it.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse

import workloads as W
from oracle import krylov, models, dense
from oracle.krylov import Options
from oracle.quadrature import tanh_sinh


def random_hermitian(d, seed, density=0.05):
    u = W.uniform(seed, 4 * d * d)
    A = np.zeros((d, d), dtype=complex)
    mask = u[: d * d].reshape(d, d) < density
    A[mask] = (u[d * d: 2 * d * d].reshape(d, d)[mask] - 0.5) + 1j * (u[2 * d * d: 3 * d * d].reshape(d, d)[mask] - 0.5)
    A = A + A.conj().T + np.diag(u[3 * d * d: 3 * d * d + d])
    return scipy.sparse.csr_matrix(A)


CASES = {
    "tfim8": lambda: models.tfim_csr(W.tfim_params(8, seed=21)).to_scipy(),
    "xxzdm8": lambda: models.xxzdm_csr(W.xxzdm_params(8, seed=22)).to_scipy(),
    "bose5_3": lambda: models.bose_csr(W.bose_params(5, 3, seed=23)).to_scipy(),
    "random300": lambda: random_hermitian(300, 24),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("t,tol,m", [(10.0, 1e-8, 40), (3.0, 1e-6, 12), (-7.0, 1e-10, 30)])
def test_against_dense_definition(name, t, tol, m):
    H = CASES[name]()
    d = H.shape[0]
    v0 = W.random_state(31, d)
    res = krylov.evolve(H, v0, t, tol, m)
    assert res.status == "ok"
    assert res.t_reached == t
    ref = dense.expm_apply(H, v0, t)
    err = np.linalg.norm(res.v - ref)
    assert err <= res.err_bound + 1e-12
    assert res.err_bound <= tol * (1 + 1e-12)


@pytest.mark.parametrize("quad,reorth", [("gauss", False), ("tanh-sinh", True), ("gauss", True)])
def test_options_against_dense(quad, reorth):
    H = CASES["xxzdm8"]()
    v0 = W.random_state(32, H.shape[0])
    res = krylov.evolve(H, v0, 6.0, 1e-8, 25, Options(quad=quad, reorth=reorth))
    ref = dense.expm_apply(H, v0, 6.0)
    assert np.linalg.norm(res.v - ref) <= res.err_bound + 1e-12
    assert res.err_bound <= 1e-8 * (1 + 1e-12)


def test_rabi_closed_form_with_breakdown():
    """Two-level system: exp(-iHt) = cos(w t) I - i sin(w t) H / w, w = sqrt(D^2 + O^2) / 2."""
    D, O = 0.7, 1.3
    H = scipy.sparse.csr_matrix(0.5 * np.array([[D, O], [O, -D]], dtype=complex))
    v0 = np.array([1.0, 0.0], dtype=complex)
    for t in [0.3, 5.0, 40.0]:
        w = 0.5 * math.hypot(D, O)
        exact = math.cos(w * t) * v0 - 1j * math.sin(w * t) / w * (H @ v0)
        res = krylov.evolve(H, v0, t, 1e-8, 40)
        assert res.breakdowns == 1 and res.restarts == 1 and res.matvecs == 2
        assert np.linalg.norm(res.v - exact) <= 1e-12


def test_decoupled_spins_closed_form():
    """TFIM with J = 0: each spin rotates, exp(i h_i t sigma^x_i) on |up...up>."""
    L = 10
    p = W.tfim_params(L, seed=25)
    p["J"] = np.zeros(L - 1)
    H = models.tfim_csr(p).to_scipy()
    t = 3.0
    v0 = W.basis_state(1 << L, 0)
    res = krylov.evolve(H, v0, t, 1e-9, 30)
    r = np.arange(1 << L)
    exact = np.ones(1 << L, dtype=complex)
    for i in range(L):
        bit = (r >> i) & 1
        exact *= np.where(bit == 0, math.cos(p["h"][i] * t), 1j * math.sin(p["h"][i] * t))
    assert np.linalg.norm(res.v - exact) <= res.err_bound + 1e-12
    assert res.err_bound <= 1e-9


def test_one_boson_against_coupling_matrix_exponential():
    K = 14
    p = W.bose_params(K, 1, seed=4)
    H = models.bose_csr(p).to_scipy()
    C = H.toarray()
    v0 = W.basis_state(K, 0)
    res = krylov.evolve(H, v0, 20.0, 1e-10, 50)
    exact = scipy.linalg.expm(-1j * 20.0 * C) @ v0          # Pade, not eigh
    assert np.linalg.norm(res.v - exact) <= 1e-10 + 1e-12
    # d = 14 < m: with an orthogonal basis the 15th vector vanishes (lucky breakdown);
    # the three-term recurrence alone leaves roundoff above tol_rate there
    res = krylov.evolve(H, v0, 20.0, 1e-10, 50, Options(reorth=True))
    assert res.breakdowns == 1 and res.restarts == 1
    assert np.linalg.norm(res.v - exact) <= 1e-10 + 1e-12


def test_t_zero_and_underflow():
    H = CASES["tfim8"]()
    v0 = W.random_state(33, H.shape[0])
    res = krylov.evolve(H, v0, 0.0, 1e-8, 40)
    assert np.array_equal(res.v, v0) and res.restarts == 0
    # m = 1: the integrand is the constant h, so no step meets the rate bound
    res = krylov.evolve(H, v0, 1.0, 1e-8, 1)
    assert res.status == "step_underflow"


def test_lanczos_galerkin_relations():
    """V^H V = I (with reorthogonalisation) and H V_m = V_m H_m + h v_{m+1} e_m^T (eq. hessenbergEquation)."""
    H = CASES["random300"]()
    v0 = W.random_state(34, 300)
    m = 20
    V, a, b, h, beta0, brk = krylov.lanczos(H, v0, m + 1, 0.0, reorth=True)
    assert not brk and abs(beta0 - 1) < 1e-14
    Vm = V[:m].T                                      # d x m
    T = np.diag(a[:m]) + np.diag(b[: m - 1], 1) + np.diag(b[: m - 1], -1)
    assert np.linalg.norm(Vm.conj().T @ Vm - np.eye(m)) < 1e-13
    R = H @ Vm - Vm @ T
    R[:, m - 1] -= b[m - 1] * V[m]                    # h_{m+1,m} v_{m+1} e_m^T
    assert np.linalg.norm(R) < 1e-12 * scipy.sparse.linalg.norm(H)
    # the three-term recurrence keeps local orthogonality too
    V3, *_ = krylov.lanczos(H, v0, 6, 0.0)
    G = V3.conj() @ V3.T
    assert np.linalg.norm(G - np.eye(6)) < 1e-12


def test_error_bound_is_rigorous_without_restart():
    """||exp(-iH tau) v - V_m exp(-i H_m tau) e_1|| <= int_0^tau f (eq. errorIntegral)."""
    H = CASES["xxzdm8"]()
    v0 = W.random_state(35, H.shape[0])
    m = 12
    V, a, b, h, beta0, brk = krylov.lanczos(H, v0, m, 0.0, reorth=True)
    lam, Q = krylov.eig_hessenberg(a, b)
    f = krylov.error_integrand(lam, Q, h)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    for tau in [0.05, 0.2, 0.5, 1.0, 2.0]:
        # integrand against a Pade matrix exponential of H_m (independent of eigh)
        e = scipy.linalg.expm(-1j * tau * T)
        assert abs(f(tau)[0] - h * abs(e[m - 1, 0])) <= 1e-12 * max(1.0, h)
        approx = V.T @ krylov.krylov_exponential(lam, Q, tau)
        actual = np.linalg.norm(dense.expm_apply(H, v0, tau) - approx)
        bound, _, conv = tanh_sinh(f, 0.0, tau)
        assert conv
        assert actual <= bound * (1 + 2e-3) + 1e-14
        assert bound < 50 * actual + 1e-12          # and the bound is not vacuous


def test_forward_backward():
    """Sec. 5: evolve to t, then with -H back; the return error stays within 2 err_max."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_forward_backward.json")))
    assert g["printed_return_error"] <= g["printed_requested_bound"] == 2 * g["err_max"]
    p = W.xxzdm_params(10, seed=26)
    H = models.xxzdm_csr(p).to_scipy()
    v0 = W.basis_state(1 << 10, W.neel_index(10))
    tol, t = g["err_max"], g["t"]
    fwd = krylov.evolve(H, v0, t, tol, 40)
    back = krylov.evolve(H, fwd.v, -t, tol, 40)
    assert np.linalg.norm(back.v - v0) <= g["printed_requested_bound"] + 1e-12


def test_conservation_with_reorthogonalisation():
    """Norm and <H> are conserved by each Galerkin step (H_m real symmetric)."""
    H = CASES["random300"]()
    v0 = W.random_state(36, 300)
    res = krylov.evolve(H, v0, 8.0, 1e-8, 30, Options(reorth=True))
    e0 = np.vdot(v0, H @ v0).real
    e1 = np.vdot(res.v, H @ res.v).real
    assert abs(np.linalg.norm(res.v) - 1.0) < 1e-12
    assert abs(e1 - e0) < 1e-12 * krylov.norm1(H)


def test_xxz_sector_stays_exactly_zero():
    """XXZ conserves total S^z: components outside the Neel sector stay exactly 0."""
    L = 10
    p = W.xxzdm_params(L, seed=27)
    H = models.xxzdm_csr(p).to_scipy()
    v0 = W.basis_state(1 << L, W.neel_index(L))
    res = krylov.evolve(H, v0, 5.0, 1e-8, 30)
    pop = np.array([bin(r).count("1") for r in range(1 << L)])
    assert np.all(res.v[pop != L // 2] == 0)


# ---------------------------------------------------------------- step search

@pytest.mark.parametrize("first", [True, False])
def test_step_search_on_power_law(first):
    """E(a,b) = c (b^p - a^p): the largest admissible step solves c tau^p = r tau."""
    c, p_, r = 0.3, 5.0, 1e-3
    tau_star = (r / c) ** (1.0 / (p_ - 1.0))
    E = lambda a, b: c * (b ** p_ - a ** p_)
    opt = Options()
    out = krylov.step_search(E, 100.0, r, first, 0.5, opt, 1e-13)
    tau, err = out
    assert err <= r * tau
    assert abs(err - E(0, tau)) < 1e-15
    assert tau <= tau_star
    # the grow substep is at most tau / n_substeps, and one more would break the bound
    assert tau > tau_star / (1.0 + 1.0 / opt.n_substeps)


def test_step_search_clips_to_remaining_time():
    E = lambda a, b: 1e-20 * (b - a)
    tau, err = krylov.step_search(E, 0.37, 1e-9, True, None, Options(), 1e-13)
    assert tau == 0.37
    tau, err = krylov.step_search(E, 5.0, 1e-9, False, 1.0, Options(), 1e-13)
    assert tau == 5.0


def test_step_search_underflow():
    E = lambda a, b: 1.0 * (b - a)
    assert krylov.step_search(E, 1.0, 1e-9, True, None, Options(), 1e-13) is None


# ---------------------------------------------------------------- planted mistakes

def test_pin_catches_wrong_exponent_sign(monkeypatch):
    H = CASES["xxzdm8"]()
    v0 = W.random_state(37, H.shape[0])
    monkeypatch.setattr(krylov, "krylov_exponential",
                        lambda lam, Q, tau: Q @ (np.exp(1j * lam * tau) * Q[0, :]))
    res = krylov.evolve(H, v0, 2.0, 1e-8, 30)
    assert np.linalg.norm(res.v - dense.expm_apply(H, v0, 2.0)) > 1e-2


def test_pin_catches_transposed_hamiltonian():
    H = CASES["xxzdm8"]()
    v0 = W.random_state(38, H.shape[0])
    res = krylov.evolve(H.T.tocsr(), v0, 2.0, 1e-8, 30)
    assert np.linalg.norm(res.v - dense.expm_apply(H, v0, 2.0)) > 1e-2


def test_pin_catches_wrong_integrand_index():
    H = CASES["xxzdm8"]()
    v0 = W.random_state(39, H.shape[0])
    V, a, b, h, _, _ = krylov.lanczos(H, v0, 12, 0.0)
    lam, Q = krylov.eig_hessenberg(a, b)
    wrong = h * abs(np.sum(Q[0, :] * Q[0, :] * np.exp(-1j * lam * 0.5)))
    e = scipy.linalg.expm(-1j * 0.5 * (np.diag(a) + np.diag(b, 1) + np.diag(b, -1)))
    assert abs(wrong - h * abs(e[11, 0])) > 1e-3


def test_norm1_definition_and_roundoff_estimate():
    """||H||_1 = max column abs-sum (eq. numericalError); Rabi matrix by hand."""
    D, O = 0.7, -1.3
    H = scipy.sparse.csr_matrix(0.5 * np.array([[D, O], [O, -D]], dtype=complex))
    assert abs(krylov.norm1(H) - 0.5 * (abs(D) + abs(O))) < 1e-16
    A = CASES["xxzdm8"]()
    assert abs(krylov.norm1(A) - np.linalg.norm(A.toarray(), 1)) < 1e-13
    res = krylov.evolve(A, W.random_state(40, 256), 1.0, 1e-8, 20)
    per = 256 * krylov.norm1(A) * 2.0 ** -52
    assert res.roundoff_est == res.restarts * per
    assert res.warn_roundoff == any(per > s[1] for s in res.steps)
    res = krylov.evolve(A, W.random_state(40, 256), 1.0, 1e-14, 20)
    assert res.warn_roundoff


@pytest.mark.parametrize("n", [1, 2, 7, 40, 128])
def test_eigensolver_residual_and_orthogonality(n):
    """eig_hessenberg on random tridiagonals: ||T Q - Q Lambda|| <= 1e-13 ||T||,
    Q orthogonal to 1e-13, eigenvalues ascending and equal to the dense
    symmetric eigensolver's (a different LAPACK routine) to 1e-13 ||T||."""
    u = W.uniform(700 + n, 2 * n)
    alpha, beta = u[:n] * 4.0 - 2.0, u[n:2 * n - 1] + 0.1
    lam, Q = krylov.eig_hessenberg(alpha, beta)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    nt = np.linalg.norm(T, 2)
    assert np.linalg.norm(T @ Q - Q * lam, 2) <= 1e-13 * nt
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - np.linalg.eigvalsh(T))) <= 1e-13 * nt
