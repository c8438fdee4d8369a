"""The fused Lanczos loop (one cooperative kernel per restart, small d) against
the oracle and against the unfused kernels (TE_FUSED_OFF).

Both run the same steps of eq. arnoldi; only the order of the two grid-wide
sums per step differs, so both results must lie within 2 tol + 1e-12 of the
oracle's, and of each other.
"""
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


def solve(te, ctx, H, v0, t, tol, m, **opt):
    import torch
    o = te.make_options(**opt)
    out, st, _ = te.te_evolve(ctx, H, torch.from_numpy(v0).cuda(), t, tol, m, o)
    return out.cpu().numpy(), st


CASES = [
    ("tfim", W.tfim_params(12, 1), 10.0, 40),            # real table, d = 4096 (one slice per warp)
    ("xxzdm", W.xxzdm_params(14, 2), 6.0, 30),           # complex table, d = 16384 (several warps per block)
    ("bose", W.bose_params(8, 6, 4), 3.0, 40),           # ragged rows, d = 1716
    ("memory", W.memory_params(), 10.0, 40),             # the paper's system at its default size (d = 588)
    ("xxzdm17", W.xxzdm_params(17, 5), 1.0, 20),         # d = 131072: four slices per warp
]


@pytest.mark.parametrize("name,params,t,m", CASES, ids=[c[0] for c in CASES])
def test_fused_matches_oracle_and_unfused(te, ctx, name, params, t, m):
    tol = 1e-8
    H = te.te_build_model(ctx, params)
    try:
        d = te.te_matrix_info_get(H)["d"]
        v0 = W.random_state(77, d)
        vf, sf = solve(te, ctx, H, v0, t, tol, m)
        vu, su = solve(te, ctx, H, v0, t, tol, m, fused_lanczos=te.TE_FUSED_OFF)
        assert sf["fused_restarts"] == sf["restarts"] > 0
        assert su["fused_restarts"] == 0
        ref = krylov.evolve(models.build(params).to_scipy(), v0, t, tol, m)
        for v, s in ((vf, sf), (vu, su)):
            assert np.linalg.norm(v - ref.v) <= 2 * tol + 1e-12
            assert s["err_bound"] <= tol * (1 + 1e-12) and s["t_reached"] == t
        assert np.linalg.norm(vf - vu) <= 2 * tol + 1e-12
        assert sf["matvecs"] > 0
    finally:
        te.te_matrix_free(H)


def test_fused_breakdown_and_negative_time(te, ctx):
    """m above d ends each Krylov space by a lucky breakdown inside the fused
    kernel; t < 0 runs it with -H."""
    p = W.tfim_params(3, 9)                      # d = 8 < m
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(78, 8)
        v, st = solve(te, ctx, H, v0, -2.5, 1e-10, 20)
        assert st["fused_restarts"] > 0 and st["breakdowns"] > 0
        ref = krylov.evolve(models.build(p).to_scipy(), v0, -2.5, 1e-10, 20)
        assert np.linalg.norm(v - ref.v) <= 2e-10 + 1e-12
    finally:
        te.te_matrix_free(H)


def test_fused_is_deterministic_and_skipped_for_large_or_reorth(te, ctx):
    """Two fused solves agree bit for bit; above the size limit, with full
    reorthogonalisation or with the CSR kernel the unfused path runs."""
    H = te.te_build_model(ctx, W.xxzdm_params(12, 3))
    try:
        v0 = W.random_state(79, 4096)
        a, sa = solve(te, ctx, H, v0, 4.0, 1e-8, 30)
        b, sb = solve(te, ctx, H, v0, 4.0, 1e-8, 30)
        assert sa["fused_restarts"] > 0 and np.array_equal(a, b)
        _, sr = solve(te, ctx, H, v0, 4.0, 1e-8, 30, reorth=te.TE_REORTH_FULL)
        _, sc = solve(te, ctx, H, v0, 4.0, 1e-8, 30, spmv_lanes=4)
        assert sr["fused_restarts"] == 0 and sc["fused_restarts"] == 0
    finally:
        te.te_matrix_free(H)
    H = te.te_build_model(ctx, W.tfim_params(18, 4))    # d = 262144: above the limit
    try:
        v0 = W.random_state(80, 1 << 18)
        _, st = solve(te, ctx, H, v0, 0.5, 1e-8, 20)
        assert st["fused_restarts"] == 0
    finally:
        te.te_matrix_free(H)


def test_fused_option_is_validated(te, ctx):
    H = te.te_build_model(ctx, W.tfim_params(4, 1))
    try:
        with pytest.raises(te.TEError) as e:
            solve(te, ctx, H, W.random_state(81, 16), 1.0, 1e-8, 10, fused_lanczos=7)
        assert e.value.status == te.TE_ERR_INVALID_ARG
    finally:
        te.te_matrix_free(H)


def test_barrier_wait_is_bounded(te, ctx):
    """The fused loop's grid barrier: with every block present it passes; with
    one block absent the others give up after their bounded wait (about a
    second) and report TE_ERR_TIMEOUT, and the context keeps working."""
    st, n, ms = te.te_fused_barrier_check(ctx, -1)
    assert st == te.TE_OK and n > 0 and ms < 100.0
    st, n0, ms = te.te_fused_barrier_check(ctx, 0)
    assert st == te.TE_ERR_TIMEOUT and n0 == 0 and 500.0 < ms < 20000.0
    H = te.te_build_model(ctx, W.tfim_params(8, 2))
    try:
        v, s = solve(te, ctx, H, W.random_state(82, 256), 1.0, 1e-8, 20)
        assert s["fused_restarts"] > 0 and s["err_bound"] <= 1e-8
    finally:
        te.te_matrix_free(H)


def test_timed_out_fused_restart_is_rerun_unfused(te, ctx):
    """A grid barrier of the fused loop that gives up no longer fails the solve: with
    TE_OPT_TEST_FUSED_TIMEOUT one block of the first fused restart leaves before its
    first barrier, the others' bounded wait runs out, and the library restores that
    restart's starting state and runs it (and the rest of the solve) as separate
    launches.  The result equals the oracle within 2 tol + 1e-12."""
    import time
    p = W.tfim_params(12, 83)
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(84, 1 << 12)
        o = te.make_options()
        o.flags |= te.TE_OPT_TEST_FUSED_TIMEOUT
        a = time.perf_counter()
        out, st, s = te.te_evolve(ctx, H, v0, 6.0, 1e-8, 40, o)
        wall = time.perf_counter() - a
        assert s == te.TE_OK
        assert st["flags"] & te.TE_FLAG_FUSED_RETRY
        assert st["fused_restarts"] == 0 and st["restarts"] >= 2
        assert 0.5 < wall < 30.0                         # the bounded wait, then the retry
        ref = krylov.evolve(models.build(p).to_scipy(), v0, 6.0, 1e-8, 40)
        assert np.linalg.norm(out - ref.v) <= 2e-8 + 1e-12
        # the plan keeps serving fused solves afterwards
        out2, st2, _ = te.te_evolve(ctx, H, v0, 6.0, 1e-8, 40)
        assert st2["fused_restarts"] == st2["restarts"] and not (st2["flags"] & te.TE_FLAG_FUSED_RETRY)
        assert np.linalg.norm(out2 - ref.v) <= 2e-8 + 1e-12
    finally:
        te.te_matrix_free(H)
