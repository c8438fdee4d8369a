"""te_evolve_multi: independent problems (own H, v, t) advanced together.

Every problem is its own solve of Algorithm 1, so each result meets the single
solve's bar: within 2 tol + 1e-12 of the oracle and within its reported bound
of the dense exp(-iHt)v, whatever else runs in the same group.
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


def mixed_problems():
    """Models of different families and sizes, times of both signs and zero."""
    ps = [W.tfim_params(6, 70), W.tfim_params(9, 71), W.xxzdm_params(8, 72), W.xxzdm_params(10, 73),
          W.bose_params(6, 3, 74), W.memory_params(), W.tfim_params(4, 75)]
    ts = [3.0, -2.5, 7.0, 0.0, 4.0, 1.5, 12.0]
    return ps, ts


def test_multi_mixed_models_vs_oracle_and_dense(te, ctx):
    ps, ts = mixed_problems()
    tol, m = 1e-9, 24
    Hs = [te.te_build_model(ctx, p) for p in ps]
    try:
        As = [models.build(p).to_scipy() for p in ps]
        v0 = [W.random_state(1500 + i, A.shape[0]) for i, A in enumerate(As)]
        for device in (True, False):
            if device:
                import torch
                vin = [torch.from_numpy(v).cuda() for v in v0]
            else:
                vin = v0
            outs, sts, stat, s = te.te_evolve_multi(ctx, Hs, vin, ts, tol, m)
            assert s == te.TE_OK and stat == [te.TE_OK] * len(ps)
            outs = [o.cpu().numpy() if device else o for o in outs]
            for i, (A, v, t) in enumerate(zip(As, v0, ts)):
                assert sts[i]["t_reached"] == t, i
                if t == 0.0:
                    assert np.array_equal(outs[i], v)
                    continue
                ref = krylov.evolve(A, v, t, tol, m)
                assert np.linalg.norm(outs[i] - ref.v) <= 2 * tol + 1e-12, i
                exact = dense.expm_apply(A, v, t)
                assert np.linalg.norm(outs[i] - exact) <= sts[i]["err_bound"] + 1e-12, i
                assert sts[i]["m_used"] == min(m, A.shape[0])
    finally:
        for H in Hs:
            te.te_matrix_free(H)


def test_multi_same_matrix_many_vectors_and_breakdown(te, ctx):
    """One H shared by several problems; a d = 16 < m problem whose whole space
    fits one Krylov basis (the three-term recurrence leaves a 3e-10 residual
    there, above tol_rate, so the step search, not a breakdown, covers t, as in
    the oracle); a 4 x 4 problem that breaks down (h below tol_rate)."""
    p = W.xxzdm_params(9, 76)
    small = W.tfim_params(4, 77)
    H = te.te_build_model(ctx, p)
    Hs_ = te.te_build_model(ctx, small)
    M = W.uniform(64, 16, -1.0, 1.0).reshape(4, 4) + 1j * W.uniform(65, 16, -1.0, 1.0).reshape(4, 4)
    Hd = M + M.conj().T
    rows, cols = np.nonzero(np.ones((4, 4)))
    H4 = te.te_build_csr(ctx, 4, rows, cols, Hd[rows, cols])
    try:
        A = models.build(p).to_scipy()
        As = models.build(small).to_scipy()
        v = ([W.random_state(1600 + i, A.shape[0]) for i in range(5)] +
             [W.random_state(1699, 16), W.random_state(1698, 4)])
        ts = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 9.0]
        outs, sts, stat, s = te.te_evolve_multi(ctx, [H] * 5 + [Hs_, H4], v, ts, 1e-10, 30)
        assert s == te.TE_OK
        for i in range(5):
            exact = dense.expm_apply(A, v[i], ts[i])
            assert np.linalg.norm(outs[i] - exact) <= sts[i]["err_bound"] + 1e-12, i
        assert sts[5]["m_used"] == 16 and sts[5]["restarts"] == 1
        exact = dense.expm_apply(As, v[5], ts[5])
        assert np.linalg.norm(outs[5] - exact) <= sts[5]["err_bound"] + 1e-12
        assert sts[6]["m_used"] == 4 and sts[6]["breakdowns"] >= 1
        exact = dense.expm_apply(Hd, v[6], ts[6])
        assert np.linalg.norm(outs[6] - exact) <= sts[6]["err_bound"] + 1e-12
    finally:
        te.te_matrix_free(H)
        te.te_matrix_free(Hs_)
        te.te_matrix_free(H4)


def test_multi_bad_problem_alone_fails(te, ctx):
    ps = [W.tfim_params(7, 78), W.tfim_params(8, 79), W.tfim_params(6, 80)]
    Hs = [te.te_build_model(ctx, p) for p in ps]
    try:
        As = [models.build(p).to_scipy() for p in ps]
        v = [W.random_state(1700 + i, A.shape[0]) for i, A in enumerate(As)]
        v[1] = v[1] * 1.01
        outs, sts, stat, s = te.te_evolve_multi(ctx, Hs, v, [2.0, 2.0, 2.0], 1e-8, 20,
                                                allow=(te.TE_ERR_NOT_NORMALIZED,))
        assert stat == [te.TE_OK, te.TE_ERR_NOT_NORMALIZED, te.TE_OK]
        for i in (0, 2):
            exact = dense.expm_apply(As[i], v[i], 2.0)
            assert np.linalg.norm(outs[i] - exact) <= sts[i]["err_bound"] + 1e-12
    finally:
        for H in Hs:
            te.te_matrix_free(H)


def test_multi_more_than_group_and_deterministic(te, ctx):
    """300 tiny problems (groups of 256 and 44); repeated calls give identical bits."""
    H = te.te_build_model(ctx, W.tfim_params(3, 81))
    try:
        A = models.build(W.tfim_params(3, 81)).to_scipy()
        v = [W.random_state(2000 + i, 8) for i in range(300)]
        ts = list(np.linspace(0.5, 3.0, 300))
        o1, sts, stat, s = te.te_evolve_multi(ctx, [H] * 300, v, ts, 1e-10, 8)
        o2, _, _, _ = te.te_evolve_multi(ctx, [H] * 300, v, ts, 1e-10, 8)
        assert s == te.TE_OK and len(o1) == 300
        for i in range(0, 300, 37):
            exact = dense.expm_apply(A, v[i], ts[i])
            assert np.linalg.norm(o1[i] - exact) <= sts[i]["err_bound"] + 1e-12
        assert all(np.array_equal(a, b) for a, b in zip(o1, o2))
    finally:
        te.te_matrix_free(H)


def test_multi_full_size_tfim_x32(te, ctx):
    """The 32-chain workload as the benchmark runs it: norms and energies kept,
    bounds within tol, sampled problems equal to te_evolve, and the largest
    problem equal to the oracle within 2 tol + 1e-12."""
    import torch
    wl = W.workload("tfim_multi_x32")
    probs = wl["problems"]
    Hs = [te.te_build_model(ctx, q["params"]) for q in probs]
    try:
        v0 = [torch.from_numpy(W.random_state(q["v0_seed"], q["d"])).cuda() for q in probs]
        ts = [q["t"] for q in probs]
        outs, sts, stat, s = te.te_evolve_multi(ctx, Hs, v0, ts, wl["tol"], wl["m"])
        assert s == te.TE_OK
        for i in range(len(probs)):
            assert sts[i]["t_reached"] == ts[i] and sts[i]["err_bound"] <= wl["tol"] * (1 + 1e-12)
            assert abs(torch.linalg.vector_norm(outs[i]).item() - 1.0) <= 1e-9
        order = sorted(range(len(probs)), key=lambda i: probs[i]["d"])
        for i in (order[0], order[len(order) // 2], order[-1]):
            e0 = te.te_spmv(ctx, Hs[i], v0[i])[1]
            e1 = te.te_spmv(ctx, Hs[i], outs[i])[1]
            assert abs(e1 - e0) <= 1e-6 * max(1.0, abs(e0))
            single, _, _ = te.te_evolve(ctx, Hs[i], v0[i], ts[i], wl["tol"], wl["m"])
            assert torch.linalg.vector_norm(single - outs[i]).item() <= 2 * wl["tol"] + 1e-12
        # the largest problem (and, among the largest, the longest time) against the oracle
        big = max(range(len(probs)), key=lambda i: (probs[i]["d"], probs[i]["t"]))
        q = probs[big]
        ref = krylov.evolve(models.build(q["params"]).to_scipy(), v0[big].cpu().numpy(), q["t"],
                            wl["tol"], wl["m"], threads=os.cpu_count())
        assert np.linalg.norm(outs[big].cpu().numpy() - ref.v) <= 2 * wl["tol"] + 1e-12
    finally:
        for H in Hs:
            te.te_matrix_free(H)
