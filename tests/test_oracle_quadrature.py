"""Pins for the oracle's quadrature (Sec. 2.3 double-exponential rule, Sec. 4 Gauss option).

Closed-form integrals and an independent adaptive Gauss-Kronrod rule (scipy quad).
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle.quadrature import tanh_sinh, gauss_legendre
from oracle.krylov import error_integrand
import workloads as W


@pytest.mark.parametrize("f,a,b,exact", [
    (np.sin, 0.0, math.pi, 2.0),
    (np.sqrt, 0.0, 1.0, 2.0 / 3.0),                 # derivative singular at 0
    (np.exp, 0.0, 2.0, math.e ** 2 - 1.0),
    (lambda x: 1.0 / (1.0 + x * x), -3.0, 5.0, math.atan(5.0) + math.atan(3.0)),
    (lambda x: np.abs(0.3 * np.exp(-1j * 1.7 * x)), 0.0, 5.0, 1.5),   # |q e^{-i lam t}| = |q|
])
def test_tanh_sinh_closed_forms(f, a, b, exact):
    val, levels, conv = tanh_sinh(f, a, b)
    assert conv
    assert abs(val - exact) <= 1e-6 * abs(exact)
    # the stop rule is a 1e-3 relative-difference test; the double-exponential
    # rule's actual error is far smaller on smooth integrands
    assert levels >= 3


def test_tanh_sinh_orientation_and_zero():
    v1, _, _ = tanh_sinh(np.cos, 0.0, 1.0)
    v2, _, _ = tanh_sinh(np.cos, 1.0, 0.0)
    assert abs(v1 + v2) < 1e-12 and abs(v1 - math.sin(1.0)) < 1e-9
    v0, _, conv = tanh_sinh(lambda x: 0.0 * x, 0.0, 3.0)
    assert v0 == 0.0 and conv
    assert tanh_sinh(np.cos, 2.0, 2.0)[0] == 0.0


def test_tanh_sinh_level_cap_flags_nonconvergence():
    # a wildly oscillating integrand on a long interval cannot meet 1e-3 in 2 levels
    val, levels, conv = tanh_sinh(lambda x: np.abs(np.sin(40.0 * x)) + 0.0, 0.0, 50.0, max_level=2)
    assert levels == 2 and not conv


def test_gauss_legendre_exact_on_polynomials():
    val, _, _ = gauss_legendre(lambda x: x ** 39, 0.0, 1.0, n=20)
    assert abs(val - 1.0 / 40.0) < 1e-14
    val, _, _ = gauss_legendre(np.sin, 0.0, math.pi, n=20)
    assert abs(val - 2.0) < 1e-13


@pytest.mark.parametrize("seed", range(6))
def test_error_integral_against_gauss_kronrod(seed):
    """Random integrands of the form h |sum_k q_k e^{-i lam_k tau}| (eq. errorIntegral)."""
    rng_u = W.uniform(1000 + seed, 64)
    m = 12
    lam = -5.0 + 10.0 * rng_u[:m]
    Q = np.linalg.qr(np.reshape(W.uniform(2000 + seed, m * m, -1, 1), (m, m)))[0]
    h = 0.5 + rng_u[m]
    f = error_integrand(lam, Q, h)
    T = 0.2 + 3.0 * rng_u[m + 1]
    ref, _ = scipy.integrate.quad(lambda x: float(f(x)[0]), 0.0, T, limit=400,
                                  epsabs=0.0, epsrel=1e-12)
    val, _, conv = tanh_sinh(f, 0.0, T)
    assert conv
    assert abs(val - ref) <= 1e-3 * ref
    # the non-adaptive Gauss option is the paper's faster, less safe rule (Sec. 4):
    # it is not held to the adaptive rule's 1e-3
    g, _, _ = gauss_legendre(f, 0.0, T, n=20)
    assert abs(g - ref) <= 1e-2 * ref
    # additivity over a split interval
    a, _, _ = tanh_sinh(f, 0.0, 0.4 * T)
    b, _, _ = tanh_sinh(f, 0.4 * T, T)
    assert abs(a + b - ref) <= 2e-3 * ref
