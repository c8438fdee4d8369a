"""CPU oracle for restarted Krylov time evolution exp(-iHt)v -- TEST INFRASTRUCTURE.

A plain, slow, fp64/complex128 restatement of the TimeEvolver method (arXiv
2205.15346): Lanczos (Sec. 2.1, eq. arnoldi), the integral error bound
(Sec. 2.2, eq. errorIntegral) evaluated by tanh-sinh quadrature (Sec. 2.3, Sec. 4),
the step-size rule (eqs. errorRate and stepSize, Algorithm 1 step 2), the Krylov
exponential (eq. krylovApproximation) and the restart (Algorithm 1 step 3), plus
the Hamiltonian builders of the synthetic workloads (Sec. 3).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline leg
and its reference arm) may import this package.  It shares no code with the CUDA
library and never imports it.  Library primitives used as single steps: scipy's
sparse matrix-vector product, numpy's vdot/norm/matmul, scipy's symmetric
tridiagonal eigensolver and numpy's Gauss-Legendre nodes.

Pins (tests/test_oracle_*.py, run without a GPU): dense eigendecomposition
exp(-iHt)v, closed forms (two-level Rabi, decoupled spins, one boson), quadrature
of closed-form integrals and against scipy's adaptive Gauss-Kronrod, brute-force
Kronecker-product Hamiltonians, conservation laws and the forward-backward check
of Sec. 5.  Parity unpinned: the exact step sequence (accept/reject decisions can
flip under different rounding of sin/cos) and the roundoff estimate's printed
value for the paper's own example (eq. numericalError, Sec. 5).
"""
from .krylov import evolve, lanczos, error_integrand, step_search, EvolveResult
from .quadrature import tanh_sinh, gauss_legendre, integrate
from . import models, dense

__all__ = [
    "evolve", "lanczos", "error_integrand", "step_search", "EvolveResult",
    "tanh_sinh", "gauss_legendre", "integrate", "models", "dense",
]
