"""te_spmv (the fused SpMV kernel in plain-product mode) against the oracle's
sparse product, element by element, for every lanes-per-row variant."""
import numpy as np
import pytest
import scipy.sparse

import workloads as W
from oracle import models

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(te):
    c = te.te_create(0)
    yield c
    te.te_destroy(c)


def check_spmv(te, ctx, H, A, seed, torch_dev=False):
    d = A.shape[0]
    x = W.complex_gaussian(seed, d)
    ref = A @ x
    if torch_dev:
        import torch
        y, dot = te.te_spmv(ctx, H, torch.from_numpy(x).cuda())
        y = y.cpu().numpy()
    else:
        y, dot = te.te_spmv(ctx, H, x)
    scale = (abs(A) @ abs(x))
    assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300)
    assert abs(dot - np.vdot(x, ref).real) <= 1e-12 * np.vdot(abs(x), scale).real
    return y


@pytest.mark.parametrize("params", [
    W.tfim_params(12, 1), W.xxzdm_params(14, 2), W.xxzdm_params(9, 3, pbc=False),
    W.bose_params(8, 6, 4), W.bose_params(12, 5, 5),
], ids=lambda p: p["model"])
def test_spmv_models(te, ctx, params):
    H = te.te_build_model(ctx, params)
    try:
        check_spmv(te, ctx, H, models.build(params).to_scipy(), 11)
        check_spmv(te, ctx, H, models.build(params).to_scipy(), 12, torch_dev=True)
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("avg", [0.5, 2.5, 9.0, 30.0, 60.0, 140.0])
def test_spmv_ragged_and_empty_rows(te, ctx, avg):
    """Random rows of very different lengths (including empty rows): every lanes variant."""
    d = 3001
    u = W.uniform(int(avg * 10) + 3, 3 * d)
    lens = np.floor(2 * avg * u[:d] ** 2).astype(np.int64)
    lens[::17] = 0
    rows = np.repeat(np.arange(d), lens)
    n = rows.size
    v = W.uniform(99, 3 * n)
    cols = (v[:n] * d).astype(np.int64)
    vals = (v[n:2 * n] - 0.5) + 1j * (v[2 * n:] - 0.5)
    csr = models.coo_to_csr(d, rows, cols, vals)
    A = csr.to_scipy()
    H = te.te_build_csr(ctx, d, rows, cols, vals)
    try:
        check_spmv(te, ctx, H, A, 13)
    finally:
        te.te_matrix_free(H)


def test_spmv_single_row(te, ctx):
    H = te.te_build_csr(ctx, 1, [0], [0], [2.5 - 1j])
    try:
        y, dot = te.te_spmv(ctx, H, np.array([1j]))
        assert y[0] == (2.5 - 1j) * 1j and dot == 2.5
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("nvals,complex_diag,expect_table,real_table", [
    (100, False, True, False),   # few distinct values, real diagonal: value-indexed copy
    (100, False, True, True),    # the same with real values: the two-DFMA product
    (None, False, False, False), # every value distinct (> 65535): full-value copy
    (100, True, False, False),   # complex diagonal: full-value copy
    (100, True, False, True),    # real off-diagonal values, complex diagonal: full-value copy
])
def test_spmv_value_table_forms(te, ctx, nvals, complex_diag, expect_table, real_table):
    """The sliced copy stores a 16-bit index into a table of distinct
    off-diagonal values when it can (with a product of two DFMA per entry when
    every one of them is real); all forms give the oracle's product."""
    d, per = 5000, 20
    offs = 1 + (W.uniform(201, per) * (d - 1)).astype(np.int64)
    offs = np.unique(offs)
    rows = np.repeat(np.arange(d), offs.size)
    cols = (rows + np.tile(offs, d)) % d
    n = rows.size
    if nvals is None:
        u = W.uniform(202, 2 * n)
        vals = (u[:n] - 0.5) + 1j * (u[n:] - 0.5)
    else:
        u = W.uniform(203, 2 * nvals)
        table = (u[:nvals] - 0.5) + (0.0 if real_table else 1j * (u[nvals:] - 0.5))
        pick = (W.uniform(204, n) * nvals).astype(np.int64)
        vals = table[pick]
    dg = W.uniform(205, 2 * d) - 0.5
    dvals = dg[:d] + (1j * dg[d:] if complex_diag else 0.0)
    rows = np.concatenate([rows, np.arange(d)])
    cols = np.concatenate([cols, np.arange(d)])
    vals = np.concatenate([vals, dvals])
    A = models.coo_to_csr(d, rows, cols, vals).to_scipy()
    H = te.te_build_csr(ctx, d, rows, cols, vals)
    try:
        info = te.te_matrix_info_get(H)
        if expect_table:
            off = A.tocoo()
            mask = off.row != off.col
            distinct = len(np.unique(np.stack([off.data[mask].real, off.data[mask].imag], 1), axis=0))
            assert 0 < info["sell_dict"] <= distinct + 64     # racing inserts may repeat a value
            assert info["sell_real"] == int(real_table)
        else:
            assert info["sell_dict"] == 0 and info["sell_real"] == 0
        check_spmv(te, ctx, H, A, 14)
        check_spmv(te, ctx, H, A, 15, torch_dev=True)
    finally:
        te.te_matrix_free(H)


@pytest.mark.parametrize("params", [
    W.tfim_params(10, 1), W.xxzdm_params(12, 2), W.bose_params(8, 5, 4), W.memory_params(),
], ids=lambda p: p["model"])
def test_model_matrices_use_value_table(te, ctx, params):
    """The built-in models have real diagonals and few distinct couplings; the
    Ising chain and the paper's example system have real ones."""
    H = te.te_build_model(ctx, params)
    try:
        info = te.te_matrix_info_get(H)
        assert info["sell_dict"] > 0
        assert info["sell_real"] == int(params["model"] in ("tfim", "memory"))
    finally:
        te.te_matrix_free(H)


def test_autotune_keeps_the_product_and_solves_exact(te, ctx):
    """te_matrix_tune only changes how work is split: the product stays within
    the bound above and a solve after tuning still matches the oracle."""
    from oracle import krylov
    p = W.xxzdm_params(12, 7)
    A = models.build(p).to_scipy()
    H = te.te_build_model(ctx, p)
    try:
        v0 = W.random_state(8, A.shape[0])
        te.te_evolve(ctx, H, v0, 2.0, 1e-9, 20)          # a cached plan exists before tuning
        ms = te.te_matrix_tune(ctx, H, 3)
        info = te.te_matrix_info_get(H)
        assert ms > 0 and info["sell_tpt"] in (1, 2, 3, 4, 6, 8)
        check_spmv(te, ctx, H, A, 16)
        out, st, _ = te.te_evolve(ctx, H, v0, 2.0, 1e-9, 20)
        assert np.linalg.norm(out - krylov.evolve(A, v0, 2.0, 1e-9, 20).v) <= 2e-9 + 1e-12
    finally:
        te.te_matrix_free(H)


def test_measure_fp64_rate_is_within_the_pipe_peak(te, ctx):
    """te_measure_fp64 executes its FMA chains: the rate is a sizeable fraction of
    the FP64 pipe's derived peak (SMs x 2 FMA lanes x 2 FLOP x maximum SM clock)
    and does not exceed it."""
    import subprocess
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", "0"], capture_output=True, text=True, timeout=30).stdout
        mhz = float(out.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pytest.skip("nvidia-smi did not report the maximum SM clock")
    peak = sms * 2 * 2 * mhz * 1e6 / 1e12
    r = te.te_measure_fp64(ctx)
    assert 0.3 * peak < r <= 1.02 * peak, (r, peak)


def test_measure_fp64_mma_rate_is_positive_and_bounded(te, ctx):
    """te_measure_fp64_mma executes its matrix instructions: a positive rate, below
    the nominal FP64 rate of the fastest FP64 tensor units of this GPU family
    (the probe decides between the two FP64 paths; it asserts neither is faster)."""
    r = te.te_measure_fp64_mma(ctx)
    v = te.te_measure_fp64(ctx)
    assert 0.0 < r < 100.0 and v > 0.0, (r, v)


@pytest.mark.parametrize("params", [W.xxzdm_params(14, 2), W.bose_params(10, 6, 4),
                                    W.xxzdm_params(5, 6)],
                         ids=["xxzdm14", "bose10_6", "xxzdm5"])
def test_staged_gather_variants_are_bitwise_the_same_product(te, ctx, params):
    """The value-indexed product taking two slices per pass, and with its gathers
    staged in shared memory two or four entries ahead (cp.async), for every
    work-item size: bitwise the product of
    the register-gather kernel, and within 1e-14 (|A||x|)_i of the oracle's.  Rows
    of the bosons (17..79 entries) and the tiny chain (w < 4) cover ragged trips."""
    H = te.te_build_model(ctx, params)
    try:
        assert te.te_matrix_info_get(H)["sell_dict"] > 0
        A = models.build(params).to_scipy()
        te.te_matrix_set_sell(ctx, H, 1, 0)
        base = check_spmv(te, ctx, H, A, 13)
        for tpt in (1, 2, 3, 4, 8):
            for trip in (0, 1, 2, 4):
                te.te_matrix_set_sell(ctx, H, tpt, trip)
                assert te.te_matrix_info_get(H)["sell_async"] == trip
                y = check_spmv(te, ctx, H, A, 13)
                assert np.array_equal(y, base), (tpt, trip)
        # a solve on each staging: bitwise the same state
        v0 = W.random_state(14, A.shape[0])
        outs = []
        for trip in (0, 1, 2, 4):
            te.te_matrix_set_sell(ctx, H, 2, trip)
            out, st, _ = te.te_evolve(ctx, H, v0, 3.0, 1e-8, 30, te.make_options(fused_lanczos=1))
            outs.append(out)
        assert all(np.array_equal(o, outs[0]) for o in outs)
        te.te_matrix_tune(ctx, H)                     # the tuner may pick any of them
        assert te.te_matrix_info_get(H)["sell_async"] in (0, 1, 2, 4)
        assert np.array_equal(check_spmv(te, ctx, H, A, 13), base)
    finally:
        te.te_matrix_free(H)


def test_set_sell_rejects_staging_for_other_forms(te, ctx):
    H = te.te_build_model(ctx, W.tfim_params(8, 1))      # real value table
    try:
        with pytest.raises(te.TEError):
            te.te_matrix_set_sell(ctx, H, 1, 2)
        with pytest.raises(te.TEError):
            te.te_matrix_set_sell(ctx, H, 9, 0)
        te.te_matrix_set_sell(ctx, H, 2, 0)
    finally:
        te.te_matrix_free(H)
