"""Pins for the oracle's createMatrix (Sec. 3): operator expressions in
creation/annihilation operators on a number-conserving basis with optional
maximal occupations (Sec. 4).

Pinned by counting (basis sizes, order), by closed-form spectra (two coupled
modes; one particle hopping on an open chain), by the dedicated bosonic
builder written independently, and by Hermiticity.
"""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import models


def test_basis_sizes_and_order():
    assert len(models.operator_basis(5, 4)) == math.comb(8, 4)
    assert len(models.operator_basis(7, 3, [1] * 7)) == math.comb(7, 3)
    caps = [2, 0, 3, 1]
    brute = sorted((t for t in itertools.product(*[range(c + 1) for c in caps]) if sum(t) == 3),
                   reverse=True)
    assert models.operator_basis(4, 3, caps) == brute


def test_two_mode_spectrum_closed_form():
    """H = g (a^dag b + b^dag a) with N bosons has eigenvalues g (N - 2k), k = 0..N."""
    g, N = 0.7, 9
    op = {"L": 2, "N": N, "caps": None,
          "terms": [(g, [(0, 1), (1, 0)]), (g, [(1, 1), (0, 0)])]}
    A = models.operator_csr(op).to_scipy().toarray()
    ev = np.sort(np.linalg.eigvalsh(A))
    assert np.allclose(ev, np.sort(g * (N - 2 * np.arange(N + 1))), atol=1e-12)


def test_one_particle_on_a_chain_closed_form():
    """One particle hopping J between neighbours of an open chain of L sites:
    eigenvalues 2 J cos(k pi / (L + 1)); with maximal occupation 1 the same."""
    L, J = 9, -1.3
    terms = []
    for i in range(L - 1):
        terms += [(J, [(i, 1), (i + 1, 0)]), (J, [(i + 1, 1), (i, 0)])]
    exact = np.sort(2 * J * np.cos(np.arange(1, L + 1) * np.pi / (L + 1)))
    for caps in (None, [1] * L):
        A = models.operator_csr({"L": L, "N": 1, "caps": caps, "terms": terms}).to_scipy().toarray()
        assert np.allclose(np.sort(np.linalg.eigvalsh(A)), exact, atol=1e-12)


def bose_terms(p):
    K = p["K"]
    terms, k = [], 0
    for i in range(K):
        for j in range(i + 1, K):
            c = complex(p["c_re"][k], p["c_im"][k])
            terms.append((c, [(i, 1), (j, 0)]))
            terms.append((c.conjugate(), [(j, 1), (i, 0)]))
            k += 1
    for i in range(K):
        terms.append((p["U"][i], [(i, 1), (i, 0), (i, 1), (i, 0)]))
    return terms


def test_reproduces_the_dedicated_bosonic_builder():
    p = W.bose_params(6, 4, 110)
    A = models.operator_csr({"L": 6, "N": 4, "caps": None, "terms": bose_terms(p)}).to_scipy()
    B = models.bose_csr(p).to_scipy()
    assert abs(A - B).max() <= 1e-14 * abs(B).max()
    assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)


def test_hermitian_with_caps_and_diagonal_always_stored():
    u = W.uniform(111, 40)
    terms = [(complex(u[0], u[1]), [(0, 1), (2, 0)]), (complex(u[0], -u[1]), [(2, 1), (0, 0)]),
             (u[2], [(1, 1), (1, 0)]), (complex(u[3], u[4]), [(0, 1), (1, 1), (3, 0), (2, 0)]),
             (complex(u[3], -u[4]), [(2, 1), (3, 1), (1, 0), (0, 0)])]
    csr = models.operator_csr({"L": 4, "N": 3, "caps": [2, 3, 1, 2], "terms": terms})
    A = csr.to_scipy()
    assert abs(A - A.conj().T).max() == 0.0
    for r in range(csr.d):
        cols, _ = csr.row(r)
        assert r in cols and np.all(np.diff(cols) > 0)
