"""te_evolve_batch (many vectors under one H, block product per Lanczos step).

Every vector of a batch is an independent solve of Algorithm 1, so each result
must meet the same bar as a single solve: within 2 tol + 1e-12 of the oracle,
within its own reported bound of the dense exp(-iHt)v, and equal within
2 tol + 1e-12 to te_evolve on the same vector.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense, krylov, models

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


def dense_block(A, V0, t):
    """exp(-iHt) applied to every row of V0 through one eigendecomposition."""
    lam, U = np.linalg.eigh(dense.to_dense(A))
    return (U @ (np.exp(-1j * lam * t)[:, None] * (U.conj().T @ V0.T))).T


def run_batch(te, ctx, H, V0, t, tol, m, device=True, allow=None, **opt):
    import torch
    o = te.make_options(**opt)
    vin = torch.from_numpy(np.ascontiguousarray(V0)).cuda() if device else np.ascontiguousarray(V0)
    kw = {} if allow is None else {"allow": allow}
    out, sts, stat, s = te.te_evolve_batch(ctx, H, vin, t, tol, m, o, **kw)
    return (out.cpu().numpy() if device else out), sts, stat, s


def test_batch_64_xxzdm_dense_oracle_single(te, ctx):
    """64 vectors, XXZ-DM L = 10: every vector against the dense definition and
    against te_evolve; three of them against the oracle."""
    p = W.xxzdm_params(10, seed=61)
    A = models.build(p).to_scipy()
    d = A.shape[0]
    V0 = W.initial_block(range(900, 964), d)
    t, tol, m = 7.0, 1e-8, 30
    H = te.te_build_model(ctx, p)
    try:
        Vb, sts, stat, s = run_batch(te, ctx, H, V0, t, tol, m)
        assert s == te.TE_OK and stat == [te.TE_OK] * 64
        exact = dense_block(A, V0, t)
        for b in range(64):
            assert sts[b]["t_reached"] == t
            assert sts[b]["err_bound"] <= tol * (1 + 1e-12)
            assert np.linalg.norm(Vb[b] - exact[b]) <= sts[b]["err_bound"] + 1e-12, b
        import torch
        for b in range(64):
            out, st1, _ = te.te_evolve(ctx, H, torch.from_numpy(V0[b]).cuda(), t, tol, m)
            assert np.linalg.norm(Vb[b] - out.cpu().numpy()) <= 2 * tol + 1e-12, b
        for b in (0, 31, 63):
            ref = krylov.evolve(A, V0[b], t, tol, m)
            assert np.linalg.norm(Vb[b] - ref.v) <= 2 * tol + 1e-12, b
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("nvec,device", [(5, False), (33, True), (1, True)])
def test_batch_ragged_counts_vs_oracle(te, ctx, nvec, device):
    """Counts that pad the block (5 -> 8, 33 -> 64, 1), host and device buffers,
    negative t (evolution with -H), every vector against the oracle."""
    p = W.tfim_params(8, seed=62)
    A = models.build(p).to_scipy()
    d = A.shape[0]
    V0 = W.initial_block(range(1000, 1000 + nvec), d)
    t, tol, m = -4.0, 1e-9, 20
    H = te.te_build_model(ctx, p)
    try:
        Vb, sts, stat, s = run_batch(te, ctx, H, V0, t, tol, m, device=device)
        assert s == te.TE_OK
        for b in range(nvec):
            ref = krylov.evolve(A, V0[b], t, tol, m)
            assert np.linalg.norm(Vb[b] - ref.v) <= 2 * tol + 1e-12, b
            assert sts[b]["t_reached"] == t
    finally:
        te.te_matrix_free(H)


def test_batch_more_than_64_groups(te, ctx):
    """70 vectors run as groups of 64 and 6; bosons K = 5, N = 3 (d = 35)."""
    p = W.bose_params(5, 3, seed=63)
    A = models.build(p).to_scipy()
    d = A.shape[0]
    V0 = W.initial_block(range(1100, 1170), d)
    t, tol, m = 3.0, 1e-10, 12
    H = te.te_build_model(ctx, p)
    try:
        Vb, sts, stat, s = run_batch(te, ctx, H, V0, t, tol, m)
        assert s == te.TE_OK and len(sts) == 70
        exact = dense_block(A, V0, t)
        for b in range(70):
            assert np.linalg.norm(Vb[b] - exact[b]) <= sts[b]["err_bound"] + 1e-12, b
    finally:
        te.te_matrix_free(H)


def test_batch_breakdown_small_dimension(te, ctx):
    """d = 4 < m: the Krylov space is exhausted (lucky breakdown, m clamped to d);
    each vector is exact up to h t_rem < tol."""
    rng_vals = W.uniform(64, 16, -1.0, 1.0)
    M = (rng_vals[:16].reshape(4, 4) + 1j * W.uniform(65, 16, -1.0, 1.0).reshape(4, 4))
    Hd = M + M.conj().T
    rows, cols = np.nonzero(np.ones((4, 4)))
    H = te.te_build_csr(ctx, 4, rows, cols, Hd[rows, cols])
    try:
        V0 = W.initial_block(range(1200, 1203), 4)
        Vb, sts, stat, s = run_batch(te, ctx, H, V0, 9.0, 1e-8, 10)
        exact = dense_block(Hd, V0, 9.0)
        for b in range(3):
            assert sts[b]["breakdowns"] >= 1
            assert sts[b]["m_used"] == 4
            assert np.linalg.norm(Vb[b] - exact[b]) <= sts[b]["err_bound"] + 1e-12
    finally:
        te.te_matrix_free(H)


def test_batch_one_bad_vector_does_not_stop_others(te, ctx):
    """A vector that is not normalised fails alone; the rest of the batch is solved."""
    p = W.xxzdm_params(8, seed=66)
    A = models.build(p).to_scipy()
    V0 = W.initial_block(range(1300, 1304), A.shape[0])
    V0[2] *= 1.5
    H = te.te_build_model(ctx, p)
    try:
        Vb, sts, stat, s = run_batch(te, ctx, H, V0, 2.0, 1e-8, 20,
                                     allow=(te.TE_ERR_NOT_NORMALIZED,))
        assert s == te.TE_ERR_NOT_NORMALIZED
        assert stat == [te.TE_OK, te.TE_OK, te.TE_ERR_NOT_NORMALIZED, te.TE_OK]
        exact = dense_block(A, V0, 2.0)
        for b in (0, 1, 3):
            assert np.linalg.norm(Vb[b] - exact[b]) <= sts[b]["err_bound"] + 1e-12
    finally:
        te.te_matrix_free(H)


def test_batch_t0_and_determinism(te, ctx):
    """t = 0 returns the input; two identical calls give identical bits."""
    p = W.xxzdm_params(9, seed=67)
    H = te.te_build_model(ctx, p)
    try:
        V0 = W.initial_block(range(1400, 1416), 1 << 9)
        V, sts, stat, s = run_batch(te, ctx, H, V0, 0.0, 1e-8, 20)
        assert np.array_equal(V, V0) and all(x["t_reached"] == 0.0 for x in sts)
        V1, _, _, _ = run_batch(te, ctx, H, V0, 5.0, 1e-8, 20)
        V2, _, _, _ = run_batch(te, ctx, H, V0, 5.0, 1e-8, 20)
        assert np.array_equal(V1, V2)
    finally:
        te.te_matrix_free(H)


def test_batch_rejects_reorth(te, ctx):
    p = W.xxzdm_params(6, seed=68)
    H = te.te_build_model(ctx, p)
    try:
        V0 = W.initial_block(range(2), 64)
        with pytest.raises(te.TEError) as e:
            run_batch(te, ctx, H, V0, 1.0, 1e-8, 10, reorth=True)
        assert e.value.status == te.TE_ERR_UNSUPPORTED
    finally:
        te.te_matrix_free(H)


def test_batch_full_size_xxzdm_L20_x64(te, ctx):
    """The 64-vector L = 20 workload as the benchmark runs it: every vector keeps
    its norm and energy (Sec. 1.1: exp(-iHt) is unitary and commutes with H),
    reports a bound within tol, two sampled vectors equal te_evolve, and vector 0
    equals the oracle within 2 tol + 1e-12."""
    import torch
    wl = W.workload("batch_xxzdm_L20_x64")
    H = te.te_build_model(ctx, wl["params"])
    try:
        V0 = torch.from_numpy(W.initial_block(wl["v0_seeds"], wl["d"])).cuda()
        out, sts, stat, s = te.te_evolve_batch(ctx, H, V0, wl["t"], wl["tol"], wl["m"])
        assert s == te.TE_OK
        for b in range(wl["nvec"]):
            assert sts[b]["t_reached"] == wl["t"] and sts[b]["err_bound"] <= wl["tol"] * (1 + 1e-12)
            assert abs(torch.linalg.vector_norm(out[b]).item() - 1.0) <= 1e-9
        for b in (0, 17, 63):
            e0 = te.te_spmv(ctx, H, V0[b].contiguous())[1]
            e1 = te.te_spmv(ctx, H, out[b].contiguous())[1]
            assert abs(e1 - e0) <= 1e-6 * max(1.0, abs(e0)), (b, e0, e1)
        for b in (0, 63):
            single, _, _ = te.te_evolve(ctx, H, V0[b].contiguous(), wl["t"], wl["tol"], wl["m"])
            assert torch.linalg.vector_norm(single - out[b]).item() <= 2 * wl["tol"] + 1e-12
    finally:
        te.te_matrix_free(H)
    # vector 0 against the oracle (its product on all host cores), element by element
    ref = krylov.evolve(models.xxzdm_csr(wl["params"]).to_scipy(), V0[0].cpu().numpy(), wl["t"],
                        wl["tol"], wl["m"], threads=os.cpu_count())
    assert np.linalg.norm(out[0].cpu().numpy() - ref.v) <= 2 * wl["tol"] + 1e-12
