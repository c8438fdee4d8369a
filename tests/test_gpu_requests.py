"""te_submit / te_poll: concurrent requests give the same result as each solve
alone (within the tolerance), admission respects the memory budget and the
serving arena's space, continuous batching admits requests while others run,
cancel works, and the solo mode serves the same results."""
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


def test_continuous_batching_admits_while_running(te):
    """Continuous batching (the default): a long request is running when short
    requests arrive; they are admitted at the next restart boundary, share its
    rounds and finish long before it, and every result equals the solve alone
    within the error bound (the benchmark spec: the same alone and in the mix)."""
    import time
    ctx = te.te_create(0)
    try:
        big_p = W.xxzdm_params(20, 82)
        Hb = te.te_build_model(ctx, big_p)
        small = [(W.tfim_params(10 + i, 83 + i), 2.0 + i, (1e-6, 1e-8, 1e-10)[i % 3]) for i in range(6)]
        Hs = [te.te_build_model(ctx, p) for p, _, _ in small]
        try:
            vb = W.random_state(90, 1 << 20)
            solo_b, st_b, _ = te.te_evolve(ctx, Hb, vb, 100.0, 1e-8, 40)
            vs = [W.random_state(91 + i, 1 << (10 + i)) for i in range(len(small))]
            solo_s = [te.te_evolve(ctx, H, v, t, tol, 40)[0] for H, v, (p, t, tol) in zip(Hs, vs, small)]
            t0 = time.perf_counter()
            rb = te.te_submit(ctx, Hb, vb, 100.0, 1e-8, 40)
            time.sleep(0.05)                           # the long request is running
            rs = [te.te_submit(ctx, H, v, t, tol, 40) for H, v, (p, t, tol) in zip(Hs, vs, small)]
            done_small = []
            for r, v, ref, (p, t, tol) in zip(rs, vs, solo_s, small):
                out = np.empty_like(v)
                s, st = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK, te.te_last_error(ctx)
                done_small.append(time.perf_counter() - t0)
                assert st["t_reached"] == t and st["err_bound"] <= tol
                assert np.linalg.norm(out - ref) <= 2 * tol + 1e-12
            s, _ = te.te_poll(rb, None)
            assert s == te.TE_PENDING                 # the short ones did not wait for it
            out = np.empty_like(vb)
            s, st = te.te_wait(rb, 120000.0, out)
            assert s == te.TE_OK and st["t_reached"] == 100.0
            assert np.linalg.norm(out - solo_b) <= 2e-8 + 1e-12
            for r in rs + [rb]:
                te.te_request_free(r)
        finally:
            te.te_matrix_free(Hb)
            for H in Hs:
                te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)


def test_batched_requests_against_oracle_with_mixed_options(te):
    """Requests with different tolerances, quadratures, small-exponential methods,
    signs of t and a t = 0 request, served together in one arena, against the
    oracle within 2 tol + 1e-12; a request that is not normalised fails alone."""
    from oracle import krylov, models
    from oracle.krylov import Options
    ctx = te.te_create(0)
    try:
        jobs = [
            (W.xxzdm_params(11, 100), 5.0, 1e-8, dict(), Options()),
            (W.tfim_params(9, 101), -3.0, 1e-10, dict(quad="gauss"), Options(quad="gauss")),
            (W.bose_params(7, 4, 102), 4.0, 1e-6, dict(small_exp="eig"), Options()),
            (W.xxzdm_params(8, 103), 0.0, 1e-8, dict(), Options()),
            (W.tfim_params(12, 104), 7.5, 1e-8, dict(n_substeps=5), Options(n_substeps=5)),
        ]
        mats, reqs, refs = [], [], []
        for i, (p, t, tol, gopt, oopt) in enumerate(jobs):
            H = te.te_build_model(ctx, p)
            mats.append(H)
            A = models.build(p).to_scipy()
            v0 = W.random_state(110 + i, A.shape[0])
            refs.append((krylov.evolve(A, v0, t, tol, 30, oopt).v, tol, v0))
            reqs.append(te.te_submit(ctx, H, v0, t, tol, 30, te.make_options(**gopt)))
        bad = W.random_state(120, 1 << 11) * 1.001
        rbad = te.te_submit(ctx, mats[0], bad, 1.0, 1e-8, 30)
        try:
            for r, (ref, tol, v0) in zip(reqs, refs):
                out = np.empty_like(v0)
                s, st = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK, te.te_last_error(ctx)
                assert np.linalg.norm(out - ref) <= 2 * tol + 1e-12
            s, _ = te.te_wait(rbad, 120000.0, None)
            assert s == te.TE_ERR_NOT_NORMALIZED
        finally:
            for r in reqs + [rbad]:
                te.te_request_free(r)
            for H in mats:
                te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)


def test_small_arena_admits_by_space_and_solo_mode(te):
    """An arena with room for two 2^14-element requests serves eight of them in
    turn (admission by free space); a request larger than the arena goes to the
    solo workers; TE_SERVE_SOLO serves the same requests with the same results."""
    ctx = te.te_create(0)
    try:
        te.te_serve_config(ctx, te.TE_SERVE_BATCH, 30, 2 * (1 << 14))
        p = W.xxzdm_params(14, 130)
        H = te.te_build_model(ctx, p)
        Hbig = te.te_build_model(ctx, W.xxzdm_params(16, 131))
        try:
            vs = [W.random_state(140 + i, 1 << 14) for i in range(8)]
            solo = [te.te_evolve(ctx, H, v, 3.0, 1e-8, 30)[0] for v in vs]
            rs = [te.te_submit(ctx, H, v, 3.0, 1e-8, 30) for v in vs]
            vbig = W.random_state(150, 1 << 16)
            rbig = te.te_submit(ctx, Hbig, vbig, 2.0, 1e-8, 30)
            outs = []
            for r, v, ref in zip(rs, vs, solo):
                out = np.empty_like(v)
                s, st = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK
                assert np.linalg.norm(out - ref) <= 2e-8 + 1e-12
                outs.append(out)
            out = np.empty_like(vbig)
            s, _ = te.te_wait(rbig, 120000.0, out)
            assert s == te.TE_OK
            ref_big = te.te_evolve(ctx, Hbig, vbig, 2.0, 1e-8, 30)[0]
            assert np.array_equal(out, ref_big)        # solo worker: the same kernels
            for r in rs + [rbig]:
                te.te_request_free(r)
            with pytest.raises(te.TEError):            # the arena exists: its shape is fixed
                te.te_serve_config(ctx, te.TE_SERVE_BATCH, 40, 1 << 20)
            te.te_serve_config(ctx, te.TE_SERVE_SOLO)
            rs = [te.te_submit(ctx, H, v, 3.0, 1e-8, 30) for v in vs[:3]]
            for r, ref in zip(rs, solo[:3]):
                out = np.empty(1 << 14, dtype=np.complex128)
                s, _ = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK and np.array_equal(out, ref)
                te.te_request_free(r)
        finally:
            te.te_matrix_free(H)
            te.te_matrix_free(Hbig)
    finally:
        te.te_destroy(ctx)


def test_cancel_running_batched_request(te):
    ctx = te.te_create(0)
    try:
        H = te.te_build_model(ctx, W.xxzdm_params(16, 160))
        try:
            v = W.random_state(161, 1 << 16)
            r = te.te_submit(ctx, H, v, 2000.0, 1e-10, 40)
            import time
            time.sleep(0.2)
            te.te_cancel(r)
            s, _ = te.te_wait(r, 120000.0, None)
            assert s == te.TE_ERR_CANCELLED
            te.te_request_free(r)
            r = te.te_submit(ctx, H, v, 1.0, 1e-8, 40)   # the loop still serves
            s, st = te.te_wait(r, 120000.0, None)
            assert s == te.TE_OK and st["t_reached"] == 1.0
            te.te_request_free(r)
        finally:
            te.te_matrix_free(H)
    finally:
        te.te_destroy(ctx)


def test_large_lane_runs_large_requests_one_at_a_time(te):
    """With the large-lane threshold at 2^17 stored entries, TFIM L = 14 requests
    (245,760 entries) run one at a time as solo solves beside the batch (bitwise
    te_evolve's result, finished in arrival order), while small requests are
    batched and finish within the error bound of their solo solves."""
    import time
    ctx = te.te_create(0)
    try:
        te.te_serve_config(ctx, te.TE_SERVE_BATCH, 40, 1 << 20, 1 << 17)
        Hl = te.te_build_model(ctx, W.tfim_params(14, 170))
        Hs = te.te_build_model(ctx, W.xxzdm_params(10, 171))
        try:
            vl = [W.random_state(172 + i, 1 << 14) for i in range(3)]
            vs = [W.random_state(180 + i, 1 << 10) for i in range(6)]
            solo_l = [te.te_evolve(ctx, Hl, v, 8.0, 1e-8, 40)[0] for v in vl]
            solo_s = [te.te_evolve(ctx, Hs, v, 5.0, 1e-8, 40)[0] for v in vs]
            rl = [te.te_submit(ctx, Hl, v, 8.0, 1e-8, 40) for v in vl]
            rs = [te.te_submit(ctx, Hs, v, 5.0, 1e-8, 40) for v in vs]
            finish = []
            pending = set(range(len(rl)))
            t0 = time.perf_counter()
            while pending and time.perf_counter() - t0 < 120.0:
                for i in sorted(pending):
                    if te.te_poll(rl[i], None)[0] != te.TE_PENDING:
                        finish.append(i)
                        pending.discard(i)
                time.sleep(0.0005)
            assert finish == [0, 1, 2]                 # first come, first served
            for r, ref in zip(rl, solo_l):
                out = np.empty(1 << 14, dtype=np.complex128)
                s, _ = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK and np.array_equal(out, ref)
            for r, ref in zip(rs, solo_s):
                out = np.empty(1 << 10, dtype=np.complex128)
                s, _ = te.te_wait(r, 120000.0, out)
                assert s == te.TE_OK and np.linalg.norm(out - ref) <= 2e-8 + 1e-12
            for r in rl + rs:
                te.te_request_free(r)
        finally:
            te.te_matrix_free(Hl)
            te.te_matrix_free(Hs)
    finally:
        te.te_destroy(ctx)
