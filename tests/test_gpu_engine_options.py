"""Options of the batched, grouped and sampled engines against the oracle with
the same options: both evaluations of exp(-i H_m tau) e_1 (Chebyshev series,
diagonalisation), both quadratures, full reorthogonalisation where the engine
has it, and a solve on the full-value sliced copy."""
import numpy as np
import pytest
import scipy.sparse

import workloads as W
from oracle import krylov, models
from oracle.krylov import Options

pytestmark = pytest.mark.gpu

COMBOS = [("eig", "tanh-sinh"), ("cheb", "gauss"), ("eig", "gauss")]


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


@pytest.mark.parametrize("small_exp,quad", COMBOS)
def test_batch_options(te, ctx, small_exp, quad):
    p = W.xxzdm_params(9, 130)
    A = models.build(p).to_scipy()
    V0 = W.initial_block(range(1800, 1806), A.shape[0])
    H = te.te_build_model(ctx, p)
    try:
        o = te.make_options(small_exp=small_exp, quad=quad)
        out, sts, stat, s = te.te_evolve_batch(ctx, H, V0, -3.0, 1e-9, 20, o)
        for b in range(6):
            ref = krylov.evolve(A, V0[b], -3.0, 1e-9, 20, Options(quad=quad))
            assert np.linalg.norm(out[b] - ref.v) <= 2e-9 + 1e-12, b
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("small_exp,quad", COMBOS)
def test_multi_options(te, ctx, small_exp, quad):
    ps = [W.tfim_params(7, 131), W.xxzdm_params(8, 132), W.bose_params(5, 3, 133)]
    ts = [2.5, -1.5, 4.0]
    Hs = [te.te_build_model(ctx, p) for p in ps]
    try:
        As = [models.build(p).to_scipy() for p in ps]
        v0 = [W.random_state(1900 + i, A.shape[0]) for i, A in enumerate(As)]
        o = te.make_options(small_exp=small_exp, quad=quad)
        outs, sts, stat, s = te.te_evolve_multi(ctx, Hs, v0, ts, 1e-9, 18, o)
        for i, (A, v, t) in enumerate(zip(As, v0, ts)):
            ref = krylov.evolve(A, v, t, 1e-9, 18, Options(quad=quad))
            assert np.linalg.norm(outs[i] - ref.v) <= 2e-9 + 1e-12, i
    finally:
        for H in Hs:
            te.te_matrix_free(H)


@pytest.mark.parametrize("small_exp,quad,reorth", [("eig", "tanh-sinh", True), ("cheb", "gauss", False),
                                                   ("eig", "gauss", True)])
def test_sampled_options(te, ctx, small_exp, quad, reorth):
    p = W.xxzdm_params(9, 134)
    A = models.build(p).to_scipy()
    v0 = W.random_state(135, A.shape[0])
    ts = [0.0, 0.7, 1.9, 3.3, 5.0]
    H = te.te_build_model(ctx, p)
    try:
        o = te.make_options(small_exp=small_exp, quad=quad, reorth=reorth)
        out, samp, _, bounds, st, s = te.te_evolve_sampled(ctx, H, v0, 5.0, ts, 1e-9, 16, o)
        ref = krylov.evolve(A, v0, 5.0, 1e-9, 16, Options(quad=quad, reorth=reorth), samples=ts)
        for k in range(len(ts)):
            assert np.linalg.norm(samp[k] - ref.samples[k]) <= 2e-9 + 1e-12, k
    finally:
        te.te_matrix_free(H)


def test_solve_on_the_full_value_copy(te, ctx):
    """More than 65535 distinct off-diagonal values: the sliced copy keeps full
    values; the solve still matches the oracle."""
    d, per = 4000, 12
    u = W.uniform(136, 3 * d * per)
    rows = np.repeat(np.arange(d), per)
    cols = (rows + 1 + (u[: d * per] * (d - 1)).astype(np.int64)) % d
    vals = (u[d * per: 2 * d * per] - 0.5) + 1j * (u[2 * d * per:] - 0.5)
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(d, d))
    A = (A + A.conj().T).tocsr() + scipy.sparse.diags(W.uniform(137, d) - 0.5)
    c = A.tocoo()
    H = te.te_build_csr(ctx, d, c.row, c.col, c.data)
    try:
        assert te.te_matrix_info_get(H)["sell_dict"] == 0
        v0 = W.random_state(138, d)
        out, st, _ = te.te_evolve(ctx, H, v0, 3.0, 1e-9, 30)
        ref = krylov.evolve(A, v0, 3.0, 1e-9, 30)
        assert np.linalg.norm(out - ref.v) <= 2e-9 + 1e-12
    finally:
        te.te_matrix_free(H)
