"""Oracle: restarted Krylov evolution exp(-iHt)v, Algorithm 1 (test infrastructure only).

Written from arXiv 2205.15346, Sec. 2.  Notation follows the paper: v_j Lanczos
vectors, h_{j,j} (alpha_j here) and h_{j+1,j} (beta_j here) the entries of the
tridiagonal Hessenberg matrix H_m, h = h_{m+1,m}, tol_rate = err_max / t
(eq. errorRate), t_step the step size (eq. stepSize).

Readings where the paper is silent, garbled or ambiguous (the CUDA library
follows the same readings, written independently):

* H form.  The recurrence runs on H (eq. arnoldi) rather than A = -iH
  (Algorithm 1); the two differ by the diagonal similarity v_j -> i^(j-1) v_j,
  give the same approximation and the same |e_m^T exp(.) e_1|.  H_m is then
  real symmetric tridiagonal.
* alpha_j = Re <v_j, p> with <a, b> = sum conj(a_i) b_i; the imaginary part is
  roundoff for Hermitian H and is dropped.
* Lucky breakdown: if h_{j+1,j} < tol_rate the inner loop stops with m_eff = j
  and h = h_{j+1,j}.  Since |e^T exp(-iH_m tau) e_1| <= 1 the integrand is below
  h < tol_rate, so the step covers the whole remaining time with the bound
  err_step = h * t_rem.
* Restart normalisation: beta0 = ||w||, v_1 = w / beta0, w <- beta0 V_m omega.
* Step search (step 2): the first restart starts from t_step0 = 0.1 without the
  0.97 shrink and doubles while the doubled step passes; later restarts start
  from 0.97 * previous step.  Then halve while the error exceeds tol_rate * step,
  then grow by substeps of step / n_substeps, substep n covering
  [step + n s, step + (n+1) s], accepted while the accumulated integral stays
  within tol_rate times the new end.  "<=" accepts.  Every candidate is clipped
  to the remaining time t_rem so the solve ends exactly at t.  The grow loop takes
  at most max_substeps substeps; a step below min_step_rel * |t| is an underflow.
* Negative t evolves with -H for |t| (the H -> -H reversal of Sec. 5).
* The 1e-3 quadrature tolerance is not added to the bound (the paper calls it
  negligible, Sec. 2.3).
* Roundoff estimate d ||H||_1 eps with eps = 2^-52 (eq. numericalError), compared
  with the step's error integral at the end of step 2 of every restart (Sec. 2.4):
  the warning fires when it is the larger, and the reported estimate is its sum
  over the restarts (the paper's printed 3.2e-6 for its benchmark system matches
  this sum over ~50 restarts, not a single term).
* Optional full reorthogonalisation (not in the paper, which uses the three-term
  recurrence): classical Gram-Schmidt against v_1..v_j applied twice after the
  alpha_j subtraction; H_m keeps only alpha and beta.
* Intermediate times (the extension remarked in Sec. 2.4): a sample time s with
  t_now < |s| <= t_now + t_step (0 <= |s| in the first restart; every remaining
  sample in the restart that reaches t) is evaluated from the restart's H_m and
  V_m as beta0 V_m exp(-i H_m (|s| - t_now)) e_1.  Its reported bound is the
  accumulated bound at the end of that restart (the integrand is non-negative,
  so the error integral up to |s| is at most the step's).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse

from .quadrature import integrate

EPS = 2.0 ** -52


@dataclass
class Options:
    quad: str = "tanh-sinh"        # or "gauss"
    gauss_n: int = 20
    n_substeps: int = 10
    t_step0: float = 0.1
    shrink: float = 0.97
    quad_rel_tol: float = 1e-3
    quad_max_levels: int = 15
    max_substeps: int = 1000
    min_step_rel: float = 1e-13
    reorth: bool = False


@dataclass
class EvolveResult:
    v: np.ndarray
    status: str = "ok"             # "ok" or "step_underflow"
    t_reached: float = 0.0
    restarts: int = 0
    matvecs: int = 0
    breakdowns: int = 0
    err_bound: float = 0.0
    quad_warnings: int = 0
    roundoff_est: float = 0.0
    warn_roundoff: bool = False
    steps: list = field(default_factory=list)   # (t_step, err_step, m_eff, breakdown)
    samples: list = field(default_factory=list)  # vectors at the requested sample times
    sample_bounds: list = field(default_factory=list)


def norm1(H) -> float:
    """||H||_1 = maximum absolute column sum."""
    A = scipy.sparse.csr_matrix(H)
    colsum = np.bincount(A.indices, weights=np.abs(A.data), minlength=A.shape[1])
    return float(colsum.max()) if colsum.size else 0.0


def lanczos(H, w, m: int, tol_rate: float, sign: float = 1.0, reorth: bool = False):
    """Step 1 of Algorithm 1: Lanczos on sign*H started from w (eq. arnoldi).

    Returns (V, alpha, beta, h, beta0, breakdown) with V of shape (m_eff, d)
    holding v_1..v_{m_eff} as rows, alpha the diagonal and beta the
    off-diagonal of H_m, h = h_{m_eff+1, m_eff}.
    """
    d = w.shape[0]
    beta0 = float(np.linalg.norm(w))
    V = np.empty((m, d), dtype=np.complex128)
    alpha = np.zeros(m)
    beta = np.zeros(max(m - 1, 0))
    V[0] = w / beta0                                   # v_1 = w / ||w||
    h = 0.0
    m_eff = m
    breakdown = False
    for j in range(m):                                 # j = 0 is the paper's j = 1
        p = sign * (H @ V[j])                          # w_j = H v_j
        if j > 0:
            p = p - beta[j - 1] * V[j - 1]             # w_j -= h_{j-1,j} v_{j-1}
        alpha[j] = float(np.vdot(V[j], p).real)        # h_{j,j} = <v_j, w_j>
        p = p - alpha[j] * V[j]                        # w~_j = w_j - h_{j,j} v_j
        if reorth:
            for _ in range(2):
                p = p - V[: j + 1].T @ (V[: j + 1].conj() @ p)
        no = float(np.linalg.norm(p))                  # h_{j+1,j} = ||w~_j||
        if no < tol_rate:                              # lucky breakdown
            m_eff = j + 1
            h = no
            breakdown = True
            break
        if j < m - 1:
            beta[j] = no
            V[j + 1] = p / no                          # v_{j+1} = w~_j / h_{j+1,j}
        else:
            h = no
    return V[:m_eff], alpha[:m_eff], beta[: m_eff - 1], h, beta0, breakdown


def eig_hessenberg(alpha, beta):
    """Diagonalise the real symmetric tridiagonal H_m (done once per restart, Sec. 2.4)."""
    if len(alpha) == 1:
        return np.array(alpha, dtype=np.float64), np.ones((1, 1))
    lam, Q = scipy.linalg.eigh_tridiagonal(alpha, beta)
    return lam, Q


def error_integrand(lam, Q, h: float):
    """Integrand of eq. errorIntegral: f(tau) = h |e_m^T exp(-i H_m tau) e_1|.

    With H_m = Q diag(lam) Q^T:  e_m^T exp(-i H_m tau) e_1 = sum_k Q[m,k] Q[1,k] e^{-i lam_k tau}.
    """
    q = Q[-1, :] * Q[0, :]

    def f(tau):
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        return h * np.abs(np.exp(-1j * np.outer(tau, lam)) @ q)

    return f


def step_search(E, t_rem: float, tol_rate: float, first: bool, prev_step, opt: Options,
                min_step: float):
    """Step 2 of Algorithm 1 with the readings in the module docstring.

    E(a, b) returns the error integral over [a, b].  Returns (t_step, err_step)
    or None on step underflow.
    """
    def ok(err, tau):
        return err <= tol_rate * tau

    if first:
        tau = min(opt.t_step0, t_rem)
        err = E(0.0, tau)
        if ok(err, tau):
            while 2.0 * tau <= t_rem:
                err2 = E(0.0, 2.0 * tau)
                if not ok(err2, 2.0 * tau):
                    break
                tau, err = 2.0 * tau, err2
    else:
        tau = min(opt.shrink * prev_step, t_rem)
        err = E(0.0, tau)
    while not ok(err, tau):                            # halve until the rate bound holds
        tau = 0.5 * tau
        if tau < min_step:
            return None
        err = E(0.0, tau)
    s = tau / opt.n_substeps                           # grow in substeps
    base = tau
    n = 0
    while n < opt.max_substeps and tau < t_rem:
        end = min(base + (n + 1) * s, t_rem)
        delta = E(tau, end)
        if not ok(err + delta, end):
            break
        err += delta
        tau = end
        n += 1
    return tau, err


def krylov_exponential(lam, Q, tau: float):
    """omega = exp(-i H_m tau) e_1 = Q diag(e^{-i lam tau}) Q^T e_1 (eq. krylovApproximation)."""
    return Q @ (np.exp(-1j * lam * tau) * Q[0, :])


def evolve(H, v, t: float, tol: float, m: int, opt: Options | None = None,
           max_restarts: int | None = None, samples=None, threads: int | None = None) -> EvolveResult:
    """exp(-iHt) v by Algorithm 1 (restarted Lanczos with the integral error bound).

    H: scipy sparse (or dense) Hermitian d x d; v: normalised complex vector.
    max_restarts bounds the work for timing samples (t_reached then tells how far
    the solve got).  samples: optional times with the sign of t, |s| <= |t|,
    non-decreasing in |s|; the states at those times are returned in
    res.samples (see the module docstring).  threads: None takes scipy's
    product; a count takes the plain C product of csrmv.c on that many threads
    (the same definition; bitwise the same result for any count).
    """
    opt = opt or Options()
    v = np.asarray(v, dtype=np.complex128)
    d = v.shape[0]
    res = EvolveResult(v=v.copy())
    sabs = [abs(float(x)) for x in (samples or [])]
    res.samples = [None] * len(sabs)
    res.sample_bounds = [0.0] * len(sabs)
    per_restart = d * norm1(H) * EPS                    # eq. numericalError
    if threads is not None:
        from .native import ThreadedCSR
        H = ThreadedCSR(H, threads)
    if t == 0.0:
        for k in range(len(sabs)):
            res.samples[k] = res.v.copy()
        return res
    sign = 1.0 if t > 0 else -1.0
    T = abs(t)
    tol_rate = tol / T                                  # eq. errorRate
    min_step = opt.min_step_rel * T
    m = min(m, d)
    w = res.v
    t_now = 0.0
    first = True
    prev_step = None
    nxt = 0                                             # first sample not yet evaluated
    while t_now < T:
        if max_restarts is not None and res.restarts >= max_restarts:
            break
        t_rem = T - t_now
        V, alpha, beta, h, beta0, breakdown = lanczos(H, w, m, tol_rate, sign, opt.reorth)
        m_eff = len(alpha)
        res.matvecs += m_eff
        lam, Q = eig_hessenberg(alpha, beta)
        if breakdown:
            res.breakdowns += 1
            t_step, err_step = t_rem, h * t_rem
        else:
            f = error_integrand(lam, Q, h)

            def E(a, b):
                val, _, conv = integrate(f, a, b, opt.quad, opt.quad_rel_tol,
                                         opt.quad_max_levels, opt.gauss_n)
                if not conv:
                    res.quad_warnings += 1
                return val

            found = step_search(E, t_rem, tol_rate, first, prev_step, opt, min_step)
            if found is None:
                res.status = "step_underflow"
                res.v = w
                res.t_reached = t_now
                return res
            t_step, err_step = found
        last = t_step == t_rem
        taken = []
        while nxt < len(sabs) and (last or sabs[nxt] <= t_now + t_step):
            tau_s = max(sabs[nxt] - t_now, 0.0)
            res.samples[nxt] = beta0 * (V.T @ krylov_exponential(lam, Q, tau_s))
            taken.append(nxt)
            nxt += 1
        omega = krylov_exponential(lam, Q, t_step)
        w = beta0 * (V.T @ omega)                        # w = V_m omega (step 3)
        res.restarts += 1
        res.err_bound += err_step
        for k in taken:
            res.sample_bounds[k] = res.err_bound
        res.roundoff_est += per_restart
        res.warn_roundoff = res.warn_roundoff or per_restart > err_step
        res.steps.append((t_step, err_step, m_eff, breakdown))
        t_now = T if t_step == t_rem else t_now + t_step
        first = False
        prev_step = t_step
    res.v = w
    res.t_reached = sign * t_now
    return res
