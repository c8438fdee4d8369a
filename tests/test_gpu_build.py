"""GPU builders and te_build_csr against the oracle: bit-exact CSR arrays
(Sec. 3 matrix creation), sampled rows at the full workload sizes."""
import numpy as np
import pytest

import workloads as W
from oracle import models

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


def assert_csr_equal(got, want: models.CSR):
    rp, col, val = got
    assert np.array_equal(rp.astype(np.int64), want.rowptr)
    assert np.array_equal(col.astype(np.int64), want.col)
    # bitwise equality of real and imaginary parts
    assert np.array_equal(val.view(np.uint64), want.val.view(np.uint64))


@pytest.mark.parametrize("params", [
    W.tfim_params(2, 1), W.tfim_params(8, 2), W.tfim_params(13, 3),
    W.xxzdm_params(3, 4), W.xxzdm_params(10, 5), W.xxzdm_params(11, 6, pbc=False),
    W.xxzdm_params(14, 7, delta=-1.3),
    W.bose_params(2, 1, 8), W.bose_params(6, 4, 9), W.bose_params(10, 5, 10), W.bose_params(5, 15, 11),
], ids=lambda p: f"{p['model']}")
def test_model_csr_bitexact(te, ctx, params):
    H = te.te_build_model(ctx, params)
    try:
        assert_csr_equal(te.te_matrix_export(ctx, H), models.build(params))
        info = te.te_matrix_info_get(H)
        ref = models.build(params)
        assert info["nnz"] == ref.nnz and info["d"] == ref.d
        from oracle.krylov import norm1
        assert abs(info["norm1"] - norm1(ref.to_scipy())) <= 1e-13 * info["norm1"]
        assert info["max_row_nnz"] == int(np.diff(ref.rowptr).max())
    finally:
        te.te_matrix_free(H)


def _sample_rows(d, n, seed):
    r = (W.uniform(seed, n) * d).astype(np.int64)
    return np.unique(np.concatenate([r, [0, d - 1, d // 2]]))


def test_xxzdm_L22_full_size_sampled_rows(te, ctx):
    """The 4,194,304-dimensional XXZ-DM workload: sampled rows bit-exact, nnz = d (L+2)/2."""
    wl = W.workload("xxzdm_L22")
    p = wl["params"]
    H = te.te_build_model(ctx, p)
    try:
        rp, col, val = te.te_matrix_export(ctx, H)
        d = wl["d"]
        assert rp[-1] == d * (22 + 2) // 2 == 50331648
        for r in _sample_rows(d, 300, 77):
            c, v = models.spin_row(p, int(r))
            b, e = rp[r], rp[r + 1]
            assert np.array_equal(col[b:e].astype(np.int64), c)
            assert np.array_equal(val[b:e].view(np.uint64), v.view(np.uint64))
    finally:
        te.te_matrix_free(H)


def test_bose_K14_N10_full_size_sampled_rows(te, ctx):
    """C(23,10) = 1,144,066 states; rows of 14..131 entries; sampled rows bit-exact."""
    wl = W.workload("bose_K14_N10")
    p = wl["params"]
    basis = models.BoseBasis(14, 10)
    H = te.te_build_model(ctx, p)
    try:
        rp, col, val = te.te_matrix_export(ctx, H)
        d = wl["d"]
        assert len(rp) == d + 1 == len(basis) + 1
        lens = np.diff(rp)
        assert lens.min() == 14 and lens.max() == 131
        for r in _sample_rows(d, 200, 78):
            c, v = models.bose_row(p, basis, int(r))
            b, e = rp[r], rp[r + 1]
            assert np.array_equal(col[b:e].astype(np.int64), c)
            assert np.array_equal(val[b:e].view(np.uint64), v.view(np.uint64))
        occ = wl["v0"][1]
        assert te.te_model_basis_index(p, occ) == basis.index[occ]
    finally:
        te.te_matrix_free(H)


def test_build_csr_matches_oracle_coo(te, ctx):
    d = 50
    n = 400
    u = W.uniform(90, 4 * n)
    rows = (u[:n] * d).astype(np.int64)
    cols = (u[n:2 * n] * d).astype(np.int64)
    vals = (u[2 * n:3 * n] - 0.5) + 1j * (u[3 * n:] - 0.5)
    H = te.te_build_csr(ctx, d, rows, cols, vals)
    try:
        assert_csr_equal(te.te_matrix_export(ctx, H), models.coo_to_csr(d, rows, cols, vals))
    finally:
        te.te_matrix_free(H)
    # duplicates are added in input order: (1e16 + 1) - 1e16 == 0
    H = te.te_build_csr(ctx, 3, [1, 0, 1, 2, 1], [2, 0, 2, 1, 2], [1e16, 5.0, 1.0, 7.0, -1e16])
    try:
        rp, col, val = te.te_matrix_export(ctx, H)
        assert list(rp) == [0, 1, 2, 3] and list(col) == [0, 2, 1] and val[1] == 0
    finally:
        te.te_matrix_free(H)
    # CSR input with empty rows
    H = te.te_build_csr(ctx, 4, [0, 1, 1, 1, 2], [3, 0], [2.0, 2.0], te.TE_INPUT_IS_CSR)
    try:
        rp, col, val = te.te_matrix_export(ctx, H)
        assert list(rp) == [0, 1, 1, 1, 2] and list(col) == [3, 0]
    finally:
        te.te_matrix_free(H)


def test_build_csr_errors(te, ctx):
    with pytest.raises(te.TEError) as e:
        te.te_build_csr(ctx, 3, [0, 3], [0, 0], [1.0, 1.0])
    assert e.value.status == te.TE_ERR_INVALID_ARG
    with pytest.raises(te.TEError) as e:
        te.te_build_csr(ctx, 3, [0], [0], [np.nan])
    assert e.value.status == te.TE_ERR_NONFINITE
    with pytest.raises(te.TEError) as e:
        te.te_build_csr(ctx, 2, [0, 1], [1, 0], [1j, 1j], te.TE_CHECK_HERMITIAN)
    assert e.value.status == te.TE_ERR_NOT_HERMITIAN
    H = te.te_build_csr(ctx, 2, [0, 1], [1, 0], [1j, -1j], te.TE_CHECK_HERMITIAN)
    te.te_matrix_free(H)
    with pytest.raises(te.TEError) as e:
        te.te_build_model(ctx, {**W.bose_params(4, 2, 1), "N": 16})
    assert e.value.status == te.TE_ERR_INVALID_ARG
