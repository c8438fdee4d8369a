"""Dense definition of the time evolution (test infrastructure only).

v(t) = exp(-iHt) v(0) (Sec. 1.1, eq. vOfT), computed from the Hermitian
eigendecomposition H = U diag(lam) U^H for small d, and the plain Krylov
approximation V_m exp(-i H_m t) e_1 without restarts (eq. krylovApproximation)
for checking the error bound of eq. errorIntegral directly.
"""
from __future__ import annotations

import numpy as np


def to_dense(H) -> np.ndarray:
    return H.toarray() if hasattr(H, "toarray") else np.asarray(H)


def expm_apply(H, v, t: float) -> np.ndarray:
    """exp(-iHt) v by dense Hermitian eigendecomposition."""
    A = to_dense(H)
    lam, U = np.linalg.eigh(A)
    return U @ (np.exp(-1j * lam * t) * (U.conj().T @ np.asarray(v, dtype=np.complex128)))
