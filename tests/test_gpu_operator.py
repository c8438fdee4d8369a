"""te_build_operator (createMatrix of Sec. 3 on the device) against the oracle:
CSR bit-exact, basis indices and occupations exact, solves within 2 tol."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import krylov, models

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


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
        terms.append((float(p["U"][i]), [(i, 1), (i, 0), (i, 1), (i, 0)]))
    return terms


def random_op():
    u = W.uniform(120, 64)
    terms = [(complex(u[0], u[1]), [(0, 1), (2, 0)]), (complex(u[0], -u[1]), [(2, 1), (0, 0)]),
             (u[2], [(1, 1), (1, 0)]), (complex(u[3], u[4]), [(0, 1), (1, 1), (3, 0), (2, 0)]),
             (complex(u[3], -u[4]), [(2, 1), (3, 1), (1, 0), (0, 0)]), (u[5], []),
             (u[6], [(3, 1), (3, 1), (3, 0), (3, 0)])]
    return {"L": 4, "N": 5, "caps": [3, 4, 2, 3], "terms": terms}


def chain_op(L, N, caps):
    terms = []
    for i in range(L - 1):
        terms += [(-1.0, [(i, 1), (i + 1, 0)]), (-1.0, [(i + 1, 1), (i, 0)])]
    for i in range(L):
        terms.append((0.3 * (i % 3), [(i, 1), (i, 0)]))
    return {"L": L, "N": N, "caps": caps, "terms": terms}


OPS = {
    "two_modes": lambda: {"L": 2, "N": 11, "caps": None,
                          "terms": [(0.7, [(0, 1), (1, 0)]), (0.7, [(1, 1), (0, 0)])]},
    "random_caps": random_op,
    "bose_6_4": lambda: {"L": 6, "N": 4, "caps": None, "terms": bose_terms(W.bose_params(6, 4, 121))},
    "hardcore_chain": lambda: chain_op(12, 5, [1] * 12),
    "soft_chain": lambda: chain_op(7, 6, [2] * 7),
}


@pytest.mark.parametrize("name", list(OPS))
def test_csr_bit_exact(te, ctx, name):
    op = OPS[name]()
    ref = models.operator_csr(op)
    H = te.te_build_operator(ctx, op)
    try:
        info = te.te_matrix_info_get(H)
        assert info["d"] == ref.d and info["nnz"] == ref.nnz
        rp, col, val = te.te_matrix_export(ctx, H)
        assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
        assert np.array_equal(val.view(np.float64), ref.val.view(np.float64))
    finally:
        te.te_matrix_free(H)


def test_basis_index_and_occupations(te, ctx):
    op = random_op()
    states = models.operator_basis(op["L"], op["N"], op["caps"])
    for i, s in enumerate(states):
        assert te.te_operator_basis_index(op, s) == i
    for l in range(op["L"]):
        occ = te.te_operator_occupation(ctx, op, l, len(states))
        assert np.array_equal(occ, np.array([s[l] for s in states], dtype=float))
    with pytest.raises(te.TEError):
        te.te_operator_basis_index(op, (1, 1, 1, 1))          # wrong total


def test_evolve_operator_matrix_vs_oracle(te, ctx):
    op = chain_op(10, 4, [2] * 10)
    A = models.operator_csr(op).to_scipy()
    v0 = W.random_state(122, A.shape[0])
    H = te.te_build_operator(ctx, op)
    try:
        out, st, _ = te.te_evolve(ctx, H, v0, 5.0, 1e-9, 30)
        ref = krylov.evolve(A, v0, 5.0, 1e-9, 30)
        assert np.linalg.norm(out - ref.v) <= 2e-9 + 1e-12
    finally:
        te.te_matrix_free(H)


def test_rejected_operators(te, ctx):
    bad_mode = {"L": 3, "N": 2, "caps": None, "terms": [(1.0, [(3, 1), (0, 0)])]}
    with pytest.raises(te.TEError) as e:
        te.te_build_operator(ctx, bad_mode)
    assert e.value.status == te.TE_ERR_INVALID_ARG
    many = {"L": 3, "N": 2, "caps": None, "terms": [(1.0, [(0, 1), (0, 0)])] * 300}
    with pytest.raises(te.TEError) as e:
        te.te_build_operator(ctx, many)
    assert e.value.status == te.TE_ERR_UNSUPPORTED


def test_bosons_at_config_size_match_the_dedicated_builder(te, ctx):
    """14 modes, 10 bosons (d = 1,144,066): the generic builder and the dedicated
    bosonic builder give the same matrix (same pattern, values within rounding:
    the dedicated builder takes sqrt(n_j) sqrt(n_i + 1), the generic one
    sqrt(n_j (n_i + 1)))."""
    import torch
    p = W.bose_params(14, 10, 4)
    Hg = te.te_build_operator(ctx, {"L": 14, "N": 10, "caps": None, "terms": bose_terms(p)})
    Hb = te.te_build_model(ctx, p)
    try:
        ig, ib = te.te_matrix_info_get(Hg), te.te_matrix_info_get(Hb)
        assert ig["d"] == ib["d"] == math.comb(23, 10) and ig["nnz"] == ib["nnz"]
        x = torch.from_numpy(W.complex_gaussian(123, ig["d"])).cuda()
        yg, _ = te.te_spmv(ctx, Hg, x)
        yb, _ = te.te_spmv(ctx, Hb, x)
        assert (torch.linalg.vector_norm(yg - yb) / torch.linalg.vector_norm(yb)).item() <= 1e-14
    finally:
        te.te_matrix_free(Hg)
        te.te_matrix_free(Hb)
