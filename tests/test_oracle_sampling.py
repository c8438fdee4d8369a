"""Pins for the oracle's intermediate-time sampling (the extension remarked in
Sec. 2.4: states at any time inside a step from that restart's H_m and V_m)
and for the occupation observables of Sec. 5.

Each pin comes from outside the oracle: a closed form (decoupled spins), the
dense definition exp(-iHt)v at every sample time, the conservation laws the
paper uses as its consistency check for the example system, and counting
identities of the number operators.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense, krylov, models


def decoupled_spins(L, seed):
    """TFIM with J = 0: H = -sum_i h_i X_i, spins precess independently."""
    p = W.tfim_params(L, seed)
    p = dict(p, J=np.zeros(L - 1))
    return p


def product_state_closed_form(h, t):
    """exp(i t sum_i h_i X_i) |up...up>: site i is cos(h_i t)|up> + i sin(h_i t)|down>
    (bit i set = down)."""
    L = len(h)
    d = 1 << L
    v = np.ones(d, dtype=np.complex128)
    idx = np.arange(d)
    for i in range(L):
        bit = (idx >> i) & 1
        v *= np.where(bit == 1, 1j * np.sin(h[i] * t), np.cos(h[i] * t))
    return v


def test_samples_match_decoupled_spins_closed_form():
    p = decoupled_spins(8, 90)
    A = models.build(p).to_scipy()
    v0 = W.basis_state(256, 0)
    ts = list(np.linspace(0.0, 9.0, 37))
    res = krylov.evolve(A, v0, 9.0, 1e-10, 10, samples=ts)
    assert res.restarts > 3                          # samples spread over several restarts
    for s, x, b in zip(ts, res.samples, res.sample_bounds):
        exact = product_state_closed_form(p["h"], s)
        assert np.linalg.norm(x - exact) <= b + 1e-12, s


@pytest.mark.parametrize("name,t", [("xxzdm8", 6.0), ("bose5_3", -3.0), ("tfim8", 4.0)])
def test_samples_within_their_bounds_of_the_dense_definition(name, t):
    build = {"xxzdm8": lambda: models.build(W.xxzdm_params(8, 22)),
             "bose5_3": lambda: models.build(W.bose_params(5, 3, 23)),
             "tfim8": lambda: models.build(W.tfim_params(8, 21))}[name]
    A = build().to_scipy()
    v0 = W.random_state(91, A.shape[0])
    sgn = 1.0 if t > 0 else -1.0
    ts = [sgn * x for x in (0.0, 0.05, 0.5, 1.0, 1.0, 2.2, abs(t) / 2, abs(t) - 1e-3, abs(t))]
    ts = sorted(ts, key=abs)
    res = krylov.evolve(A, v0, t, 1e-9, 12, samples=ts)
    for s, x, b in zip(ts, res.samples, res.sample_bounds):
        assert np.linalg.norm(x - dense.expm_apply(A, v0, s)) <= b + 1e-12, s
        assert b <= 1e-9 * (1 + 1e-12)
    assert np.array_equal(res.samples[-1], res.v)       # the last sample is the result
    assert np.linalg.norm(res.samples[0] - v0) <= 1e-14


def test_samples_at_t_zero_return_the_input():
    A = models.build(W.tfim_params(5, 92)).to_scipy()
    v0 = W.random_state(93, 32)
    res = krylov.evolve(A, v0, 0.0, 1e-8, 10, samples=[0.0, 0.0])
    assert all(np.array_equal(x, v0) for x in res.samples)


def test_occupation_counting_identities():
    for p in (W.bose_params(6, 4, 94), W.memory_params()):
        n = models.build(p).to_scipy().shape[0]
        L = p["K"] if p["model"] == "bose" else 2 + p["K"] + p["Kp"]
        occ = np.stack([models.occupation(p, l) for l in range(L)])
        assert occ.shape == (L, n)
        if p["model"] == "bose":
            assert np.all(occ.sum(0) == p["N"])
        else:
            assert np.all(occ[0] + occ[1] == p["N0"]) and np.all(occ[2:].sum(0) == p["Nm"])
    spins = models.occupation(W.xxzdm_params(6, 95), 3)
    assert np.array_equal(spins, ((np.arange(64) >> 3) & 1).astype(float))


def test_example_system_conserves_both_sector_occupations():
    """Sec. 5: N0 = <n0> + <m0> and N_m = sum of the qubit occupations stay
    constant in time (the paper's first consistency check of its figures)."""
    p = W.memory_params()
    A = models.build(p).to_scipy()
    b = models.MemoryBasis(p)
    v0 = W.basis_state(len(b), b.index(W.memory_initial_occupation(p)))
    ts = list(np.linspace(0.0, 3.0, 13))
    res = krylov.evolve(A, v0, 3.0, 1e-8, 30, samples=ts)
    L = 2 + p["K"] + p["Kp"]
    occ = np.stack([models.occupation(p, l) for l in range(L)])
    for x in res.samples:
        n = occ @ (np.abs(x) ** 2)
        assert abs(n[0] + n[1] - p["N0"]) <= 1e-9
        assert abs(n[2:].sum() - p["Nm"]) <= 1e-9
    n0 = occ @ (np.abs(res.samples[0]) ** 2)
    assert np.allclose(n0, W.memory_initial_occupation(p), atol=1e-12)
