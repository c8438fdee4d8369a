"""te_submit / te_poll: concurrent requests give the same result as each solve
alone (within the tolerance), admission respects the memory budget, cancel works."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


def test_requests_match_solo_solves(te, ctx):
    jobs = [
        (W.tfim_params(12, 70), W.random_state(71, 1 << 12), 6.0, 1e-8, 40),
        (W.xxzdm_params(14, 72), W.random_state(73, 1 << 14), 9.0, 1e-10, 30),
        (W.xxzdm_params(10, 74), W.random_state(75, 1 << 10), -4.0, 1e-6, 20),
        (W.bose_params(9, 5, 76), None, 3.0, 1e-8, 40),
        (W.tfim_params(16, 77), W.random_state(78, 1 << 16), 2.0, 1e-8, 30),
    ]
    mats, solo, reqs = [], [], []
    for p, v0, t, tol, m in jobs:
        H = te.te_build_model(ctx, p)
        d = te.te_matrix_info_get(H)["d"]
        if v0 is None:
            v0 = W.basis_state(d, 3)
        mats.append((H, v0, t, tol, m))
        out, st, _ = te.te_evolve(ctx, H, v0, t, tol, m)
        solo.append(out)
    try:
        for rep in range(2):                       # every job twice, all in flight together
            for H, v0, t, tol, m in mats:
                reqs.append(te.te_submit(ctx, H, v0, t, tol, m))
        for i, r in enumerate(reqs):
            H, v0, t, tol, m = mats[i % len(mats)]
            out = np.empty_like(v0)
            s, st = te.te_wait(r, 120000.0, out)
            assert s == te.TE_OK, te.te_last_error(ctx)
            assert st["t_reached"] == t and st["err_bound"] <= tol
            assert np.linalg.norm(out - solo[i % len(mats)]) <= tol
            s2, _ = te.te_poll(r, None)
            assert s2 == te.TE_OK
    finally:
        for r in reqs:
            te.te_request_free(r)
        for H, *_ in mats:
            te.te_matrix_free(H)


def test_budget_and_cancel(te, ctx):
    p = W.xxzdm_params(16, 80)
    H = te.te_build_model(ctx, p)
    v0 = W.random_state(81, 1 << 16)
    try:
        te.te_set_memory_budget(ctx, 1)            # forces one request at a time
        rs = [te.te_submit(ctx, H, v0, 3.0, 1e-8, 30) for _ in range(3)]
        for r in rs:
            s, st = te.te_wait(r, 120000.0, None)
            assert s == te.TE_OK
            te.te_request_free(r)
        te.te_set_memory_budget(ctx, 1 << 40)
        r = te.te_submit(ctx, H, v0, 400.0, 1e-8, 30)
        te.te_cancel(r)
        s, st = te.te_wait(r, 120000.0, None)
        assert s in (te.TE_ERR_CANCELLED, te.TE_OK)
        te.te_request_free(r)
        r = te.te_submit(ctx, H, v0, 1.0, 1e-8, 30)
        s, _ = te.te_poll(r, None)
        assert s in (te.TE_PENDING, te.TE_OK)
        te.te_request_free(r)                      # waits for it
    finally:
        te.te_matrix_free(H)
