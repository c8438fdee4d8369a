"""Pins for the oracle's Hamiltonian builders (Sec. 3): brute-force Kronecker and
Fock-space constructions, closed-form basis counts, exact Hermiticity."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import krylov, models

I2 = np.eye(2)
SZ_PAULI = np.diag([1.0, -1.0])            # bit 0 = up (+1), bit 1 = down (-1)
SX_PAULI = np.array([[0.0, 1.0], [1.0, 0.0]])
SPLUS = np.array([[0.0, 1.0], [0.0, 0.0]])   # |up><down|
SMINUS = SPLUS.T
SZ = 0.5 * SZ_PAULI


def site_op(op, i, L):
    """Operator on site i; basis index = sum_i bit_i 2^i, so site i is kron factor L-1-i."""
    return np.kron(np.kron(np.eye(1 << (L - 1 - i)), op), np.eye(1 << i))


def tfim_dense(p):
    L = p["L"]
    H = np.zeros((1 << L, 1 << L))
    for b in range(L - 1):
        H -= p["J"][b] * site_op(SZ_PAULI, b, L) @ site_op(SZ_PAULI, b + 1, L)
    for i in range(L):
        H -= p["h"][i] * site_op(SX_PAULI, i, L)
    return H


def xxzdm_dense(p):
    L = p["L"]
    nb = L if p["pbc"] else L - 1
    H = np.zeros((1 << L, 1 << L), dtype=complex)
    for b in range(nb):
        a, c = b, (b + 1) % L
        e = complex(p["hop_re"][b], p["hop_im"][b])
        H += 0.5 * e * site_op(SPLUS, a, L) @ site_op(SMINUS, c, L)
        H += 0.5 * np.conj(e) * site_op(SMINUS, a, L) @ site_op(SPLUS, c, L)
        H += p["delta"] * site_op(SZ, a, L) @ site_op(SZ, c, L)
    for i in range(L):
        H += p["hz"][i] * site_op(SZ, i, L)
    return H


def bose_dense_fock(p):
    """H in the truncated Fock space (occupations 0..N per mode), mode 0 most significant."""
    K, N = p["K"], p["N"]
    n1 = N + 1
    a = np.diag(np.sqrt(np.arange(1, n1)), k=1)     # a|n> = sqrt(n)|n-1>
    def op(o, i):
        return np.kron(np.kron(np.eye(n1 ** i), o), np.eye(n1 ** (K - 1 - i)))
    ops = [op(a, i) for i in range(K)]
    H = np.zeros((n1 ** K, n1 ** K), dtype=complex)
    k = 0
    for i in range(K):
        for j in range(i + 1, K):
            c = complex(p["c_re"][k], p["c_im"][k])
            k += 1
            H += c * ops[i].T @ ops[j] + np.conj(c) * ops[j].T @ ops[i]
    for i in range(K):
        n_op = ops[i].T @ ops[i]
        H += p["U"][i] * n_op @ n_op
    return H


def dense_of(csr):
    return csr.to_scipy().toarray()


def assert_hermitian_bitwise(csr):
    A = csr.to_scipy().tocoo()
    lookup = {(int(r), int(c)): v for r, c, v in zip(A.row, A.col, A.data)}
    for (r, c), v in lookup.items():
        w = lookup[(c, r)]
        assert w.real == v.real and w.imag == -v.imag, (r, c)


def assert_sorted_rows(csr):
    for r in range(csr.d):
        cols, _ = csr.row(r)
        assert np.all(np.diff(cols) > 0)
        assert r in cols                               # diagonal always stored


@pytest.mark.parametrize("L", [2, 5, 7])
def test_tfim_against_kronecker(L):
    p = W.tfim_params(L, seed=11)
    csr = models.tfim_csr(p)
    assert csr.nnz == (L + 1) << L
    np.testing.assert_allclose(dense_of(csr), tfim_dense(p), atol=1e-14, rtol=0)
    assert_sorted_rows(csr)
    assert_hermitian_bitwise(csr)


@pytest.mark.parametrize("L,pbc", [(3, True), (6, True), (7, False), (8, True)])
def test_xxzdm_against_kronecker(L, pbc):
    p = W.xxzdm_params(L, seed=12, pbc=pbc)
    csr = models.xxzdm_csr(p)
    np.testing.assert_allclose(dense_of(csr), xxzdm_dense(p), atol=1e-14, rtol=0)
    assert_sorted_rows(csr)
    assert_hermitian_bitwise(csr)
    if pbc:
        # every row: diagonal + one entry per antiparallel bond; averaged over all
        # states that is 1 + L/2 exactly
        assert csr.nnz == (1 << L) * (L + 2) // 2


def test_xxzdm_rows_entrywise_match_vectorised():
    p = W.xxzdm_params(10, seed=13)
    csr = models.xxzdm_csr(p)
    for r in [0, 1, 341, 682, 1023, 517]:
        c1, v1 = csr.row(r)
        c2, v2 = models.spin_row(p, r)
        assert np.array_equal(c1, c2) and np.array_equal(v1, v2)
    pt = W.tfim_params(9, seed=14)
    csrt = models.tfim_csr(pt)
    for r in [0, 5, 511, 300]:
        c1, v1 = csrt.row(r)
        c2, v2 = models.spin_row(pt, r)
        assert np.array_equal(c1, c2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("K,N", [(2, 3), (3, 2), (4, 3), (5, 2)])
def test_bose_against_fock_space(K, N):
    p = W.bose_params(K, N, seed=15)
    basis = models.BoseBasis(K, N)
    csr = models.bose_csr(p, basis)
    Hf = bose_dense_fock(p)
    n1 = N + 1
    idx = [sum(n * n1 ** (K - 1 - i) for i, n in enumerate(s)) for s in basis.states]
    np.testing.assert_allclose(dense_of(csr), Hf[np.ix_(idx, idx)], atol=1e-13, rtol=0)
    assert_sorted_rows(csr)
    assert_hermitian_bitwise(csr)
    occ = [sum(1 for n in s if n) for s in basis.states]
    assert np.array_equal(np.diff(csr.rowptr), 1 + np.array(occ) * (K - 1))


def test_one_boson_is_the_coupling_matrix():
    """N = 1: basis index k is mode k occupied, H = C + diag(U) exactly."""
    K = 14
    p = W.bose_params(K, 1, seed=4)
    csr = models.bose_csr(p)
    C = np.zeros((K, K), dtype=complex)
    k = 0
    for i in range(K):
        for j in range(i + 1, K):
            C[i, j] = complex(p["c_re"][k], p["c_im"][k])
            C[j, i] = np.conj(C[i, j])
            k += 1
    C += np.diag(p["U"])
    assert np.array_equal(dense_of(csr), C)


def test_bose_basis_order_and_size():
    states = models.bose_basis(4, 3)
    assert states[0] == (3, 0, 0, 0) and states[-1] == (0, 0, 0, 3)
    assert all(a > b for a, b in zip(states, states[1:]))       # strictly descending lex
    assert len(states) == math.comb(6, 3)


@pytest.mark.slow
def test_bose_basis_size_config():
    """C(23, 10) = 1,144,066 states for 14 modes holding 10 bosons."""
    b = models.BoseBasis(14, 10)
    assert len(b) == 1144066 == W.bose_dim(14, 10)
    assert b.index[tuple([1] * 10 + [0] * 4)] < len(b)
    assert len(b.index) == len(b)


def test_coo_to_csr_duplicates_in_input_order():
    # (1e16 + 1) - 1e16 = 0 in binary64 when added left to right; any other order gives 1 or 2
    d = 3
    rows = [1, 0, 1, 2, 1]
    cols = [2, 0, 2, 1, 2]
    vals = [1e16, 5.0, 1.0, 7.0, -1e16]
    csr = models.coo_to_csr(d, rows, cols, vals)
    assert list(csr.rowptr) == [0, 1, 2, 3]
    assert list(csr.col) == [0, 2, 1]
    assert csr.val[1] == 0.0
    # explicit zeros are kept, empty rows allowed
    csr = models.coo_to_csr(4, [3, 0], [3, 0], [0.0, 1.0])
    assert list(csr.rowptr) == [0, 1, 1, 1, 2] and csr.val[1] == 0.0


@pytest.mark.parametrize("K,N", [(6, 4), (8, 5), (10, 5), (14, 1)])
def test_bose_vectorised_builder_is_bitwise_the_row_builder(K, N):
    """bose_csr_vec (array form, used at full size) equals bose_csr row by row, bit for bit."""
    p = W.bose_params(K, N, seed=60 + K)
    a, b = models.bose_csr(p), models.bose_csr_vec(p)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))


def test_bose_vectorised_builder_full_size_sampled_rows():
    """Config 4 size (K = 14, N = 10, d = 1,144,066): sampled rows of the array
    form equal bose_row bit for bit, and the row lengths span 14..131."""
    wl = W.workload("bose_K14_N10")
    b = models.bose_csr_vec(wl["params"])
    assert b.d == 1144066 and b.nnz == 91674506
    lens = np.diff(b.rowptr)
    assert lens.min() == 14 and lens.max() == 131
    basis = models.BoseBasis(14, 10)
    for r in (0, 1, 777, 123456, 654321, b.d - 2, b.d - 1):
        c, v = models.bose_row(wl["params"], basis, r)
        lo, hi = b.rowptr[r], b.rowptr[r + 1]
        assert np.array_equal(c, b.col[lo:hi])
        assert np.array_equal(v.view(np.uint64), b.val[lo:hi].view(np.uint64))


@pytest.mark.parametrize("kw", [{}, {"K": 6, "Kp": 6, "N0": 30, "Nm": 3, "Nc": 30.0}])
def test_memory_vectorised_builder_is_bitwise_the_row_builder(kw):
    p = W.memory_params(**kw)
    a, b = models.memory_csr(p), models.memory_csr_vec(p)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))


def test_threaded_product_is_the_plain_product():
    """The oracle's C product (csrmv.c) on 1 and 4 threads: bitwise the same, and
    equal to scipy's product to rounding (1e-15 (|A||x|)_i)."""
    from oracle import native
    A = models.build(W.bose_params(8, 5, seed=70)).to_scipy()
    x = W.complex_gaussian(71, A.shape[0])
    y1 = native.ThreadedCSR(A, 1) @ x
    y4 = native.ThreadedCSR(A, 4) @ x
    assert np.array_equal(y1, y4)
    assert np.all(np.abs(y1 - A @ x) <= 1e-15 * (abs(A) @ np.abs(x)))
    r1 = krylov.evolve(A, W.random_state(72, A.shape[0]), 3.0, 1e-8, 20, threads=1)
    r4 = krylov.evolve(A, W.random_state(72, A.shape[0]), 3.0, 1e-8, 20, threads=4)
    assert np.array_equal(r1.v, r4.v)


def test_random_hermitian_coo_is_hermitian_with_distinct_values():
    """The general-input workload: exactly Hermitian (H[j,i] = conj(H[i,j]) bit for bit),
    the flip-flop pattern of a periodic chain (L/2 off-diagonal entries per row on
    average, L + 1 stored per row at most), and one distinct value per coupled pair."""
    import scipy.sparse
    L = 10
    r, c, v = W.random_hermitian_coo(L, 9)
    d = 1 << L
    A = models.coo_to_csr(d, r, c, v).to_scipy()
    D = A - A.getH()
    assert D.count_nonzero() == 0
    assert A.nnz == d + L * d // 2
    assert np.diff(A.indptr).max() <= L + 1
    off = A.data[A.indices != np.repeat(np.arange(d), np.diff(A.indptr))]
    upper = off[np.abs(off.imag) > 0]
    assert np.unique(upper).size == upper.size           # no value repeats
    assert np.all((np.abs(off) >= 0.5) & (np.abs(off) < 1.0 + 1e-15))
