"""te_evolve_sampled (states at intermediate times, Sec. 2.4) and
te_model_occupation (the mode occupations of Sec. 5) against the oracle."""
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


@pytest.mark.parametrize("params,modes", [
    (W.tfim_params(6, 100), range(6)),
    (W.xxzdm_params(7, 101), (0, 3, 6)),
    (W.bose_params(6, 4, 102), range(6)),
    (W.memory_params(), range(10)),
])
def test_occupations_bit_exact(te, ctx, params, modes):
    import torch
    for l in modes:
        ref = models.occupation(params, l)
        host = te.te_model_occupation(ctx, params, l)
        assert np.array_equal(host, ref), l
        dev = torch.empty(ref.size, dtype=torch.float64, device="cuda")
        te.te_model_occupation(ctx, params, l, out=dev)
        assert np.array_equal(dev.cpu().numpy(), ref), l


@pytest.mark.parametrize("t", [6.0, -4.5])
def test_samples_vs_oracle_and_dense(te, ctx, t):
    p = W.xxzdm_params(9, 103)
    A = models.build(p).to_scipy()
    v0 = W.random_state(104, A.shape[0])
    sg = 1.0 if t > 0 else -1.0
    ts = [sg * x for x in (0.0, 0.05, 0.5, 1.0, 1.0, 2.2, 3.0, abs(t) - 1e-3, abs(t))]
    tol, m = 1e-9, 14
    H = te.te_build_model(ctx, p)
    try:
        out, samp, _, bounds, st, s = te.te_evolve_sampled(ctx, H, v0, t, ts, tol, m)
        ref = krylov.evolve(A, v0, t, tol, m, samples=ts)
        assert st["restarts"] > 2
        for k, x in enumerate(ts):
            assert np.linalg.norm(samp[k] - ref.samples[k]) <= 2 * tol + 1e-12, k
            assert np.linalg.norm(samp[k] - dense.expm_apply(A, v0, x)) <= bounds[k] + 1e-12, k
            assert 0.0 <= bounds[k] <= st["err_bound"] * (1 + 1e-15)
        assert np.array_equal(samp[-1], out)              # the last sample is the result
        assert np.linalg.norm(samp[0] - v0) <= 1e-13
        assert np.linalg.norm(out - ref.v) <= 2 * tol + 1e-12
    finally:
        te.te_matrix_free(H)


def test_example_system_observables_conserved_and_match_oracle(te, ctx):
    """Sec. 5: <n0> + <m0> = N0 and sum of qubit occupations = N_m at every
    sample; every occupation matches the oracle's."""
    import torch
    p = W.memory_params()
    A = models.build(p).to_scipy()
    b = models.MemoryBasis(p)
    v0 = W.basis_state(len(b), b.index(W.memory_initial_occupation(p)))
    L = 2 + p["K"] + p["Kp"]
    occ = np.stack([te.te_model_occupation(ctx, p, l) for l in range(L)])
    ts = list(np.linspace(0.0, 3.0, 13))
    tol, m = 1e-8, 30
    H = te.te_build_model(ctx, p)
    try:
        for device in (False, True):
            vin = torch.from_numpy(v0).cuda() if device else v0
            ob = torch.from_numpy(occ).cuda() if device else occ
            out, samp, n, bounds, st, s = te.te_evolve_sampled(ctx, H, vin, 3.0, ts, tol, m,
                                                               observables=ob, want_vectors=False)
            assert samp is None and n.shape == (13, L)
            assert np.all(np.abs(n[:, 0] + n[:, 1] - p["N0"]) <= 1e-9)
            assert np.all(np.abs(n[:, 2:].sum(1) - p["Nm"]) <= 1e-9)
            ref = krylov.evolve(A, v0, 3.0, tol, m, samples=ts)
            nref = np.stack([occ @ (np.abs(x) ** 2) for x in ref.samples])
            assert np.max(np.abs(n - nref)) <= 2 * (2 * tol + 1e-12) * p["N0"]
            assert np.allclose(n[0], W.memory_initial_occupation(p), atol=1e-12)
    finally:
        te.te_matrix_free(H)


def test_t_zero_and_rejected_times(te, ctx):
    p = W.tfim_params(5, 105)
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(106, 32)
        out, samp, _, _, st, s = te.te_evolve_sampled(ctx, H, v0, 0.0, [0.0, 0.0], 1e-8, 10)
        assert np.array_equal(out, v0) and all(np.array_equal(x, v0) for x in samp)
        for bad in ([1.0, 0.5], [-0.5], [2.5], [float("nan")]):
            with pytest.raises(te.TEError) as e:
                te.te_evolve_sampled(ctx, H, v0, 2.0, bad, 1e-8, 10)
            assert e.value.status == te.TE_ERR_INVALID_ARG
    finally:
        te.te_matrix_free(H)


def test_full_size_example_system_sampled():
    """The paper's benchmark system (K = K' = 10, N0 = Nc = 100, Nm = 5, t = 10,
    m = 40, tol = 1e-7) sampled at 50 times with all 22 occupations, as the
    benchmark runs it: both conservation laws at every sample, the last sample
    equals the result, the bounds never exceed tol."""
    import torch
    from paper_2205_15346_gb300 import te as te_
    c = te_.te_create(0)
    try:
        wl = W.workload("memory_K10")
        p = wl["params"]
        H = te_.te_build_model(c, p)
        L = 2 + p["K"] + p["Kp"]
        occ = torch.stack([te_.te_model_occupation(c, p, l, out=torch.empty(wl["d"], dtype=torch.float64,
                                                                             device="cuda"))
                           for l in range(L)])
        idx = te_.te_model_basis_index(p, W.memory_initial_occupation(p))
        v0 = torch.zeros(wl["d"], dtype=torch.complex128, device="cuda")
        v0[idx] = 1.0
        ts = list(np.linspace(0.0, wl["t"], 50))
        out, samp, n, bounds, st, s = te_.te_evolve_sampled(c, H, v0, wl["t"], ts, wl["tol"], wl["m"],
                                                            observables=occ)
        assert np.all(np.abs(n[:, 0] + n[:, 1] - p["N0"]) <= 1e-6)
        assert np.all(np.abs(n[:, 2:].sum(1) - p["Nm"]) <= 1e-7)
        assert torch.equal(samp[-1], out)
        assert np.all(bounds <= wl["tol"] * (1 + 1e-12))
        te_.te_matrix_free(H)
    finally:
        te_.te_destroy(c)
