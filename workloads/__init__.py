"""Seeded synthetic inputs for the Krylov time-evolution workloads.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It draws random numbers and turns them into model parameter tables
and initial vectors; it holds none of the method's arithmetic (no Lanczos, no
Hamiltonian assembly, no basis ordering, no quadrature).

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based generator:
output i of stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.
Uniforms take the top 53 bits.  Everything is plain numpy uint64/float64
arithmetic, so the tables are identical on x86 and Arm hosts.

Conventions shared by the model builders on both sides (the definitions of the
workloads, stated once here so both sides read the same words):

* spin chains: basis index bit i = 1 means spin i points down (sigma^z_i = -1),
  bit i = 0 means up;
* complex hopping amplitudes are handed over as (re, im) pairs, already formed
  from their random phases here, so the builders multiply and add only.

One workload is a general complex Hermitian matrix given as input data (COO
triplets with random values on a spin chain's sparsity pattern,
``random_hermitian_coo``); the CUDA library reads the triplets through
te_build_csr and the oracle through its own coo_to_csr.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of the counter-based splitmix64 stream ``seed`` (uint64)."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_at(seed: int, idx: np.ndarray) -> np.ndarray:
    """Outputs number idx (uint64 array) of the splitmix64 stream ``seed``."""
    i = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n uniforms on [lo, hi) from stream ``seed`` (53-bit resolution)."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def complex_gaussian(seed: int, d: int) -> np.ndarray:
    """d standard complex Gaussians (Box-Muller on 2d uniforms)."""
    u = uniform(seed, 2 * d)
    u1, u2 = u[:d], u[d:]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return r * np.cos(2.0 * np.pi * u2) + 1j * (r * np.sin(2.0 * np.pi * u2))


def random_state(seed: int, d: int) -> np.ndarray:
    """Normalised random complex128 initial vector of length d."""
    g = complex_gaussian(seed, d)
    return g / np.linalg.norm(g)


def basis_state(d: int, index: int) -> np.ndarray:
    """complex128 unit vector e_index of length d."""
    v = np.zeros(d, dtype=np.complex128)
    v[index] = 1.0
    return v


# ---------------------------------------------------------------- model tables

def tfim_params(L: int, seed: int) -> dict:
    """Transverse-field Ising chain, open boundary.

    H = -sum_{i<L-1} J_i s^z_i s^z_{i+1} - sum_i h_i s^x_i  (Pauli matrices),
    J_i, h_i ~ U[0.5, 1.5).
    """
    u = uniform(seed, 2 * L - 1, 0.5, 1.5)
    return {"model": "tfim", "L": L, "J": u[: L - 1].copy(), "h": u[L - 1:].copy()}


def xxzdm_params(L: int, seed: int, delta: float = 0.8, pbc: bool = True) -> dict:
    """XXZ chain with a Dzyaloshinskii-Moriya phase on each bond.

    H = sum_b [ 1/2 (e^{i phi_b} S^+_b S^-_{b+1} + h.c.) + delta S^z_b S^z_{b+1} ]
        + sum_i hz_i S^z_i     (spin-1/2 operators, S = sigma/2),
    phi_b ~ U[0, 2 pi), hz_i ~ U[-1, 1).  Bond b couples sites b and (b+1) mod L;
    there are L bonds with a periodic boundary, L-1 with an open one.
    """
    nb = L if pbc else L - 1
    u = uniform(seed, nb + L)
    phi = 2.0 * np.pi * u[:nb]
    return {
        "model": "xxzdm", "L": L, "pbc": bool(pbc), "delta": float(delta),
        "hop_re": np.cos(phi), "hop_im": np.sin(phi),
        "hz": -1.0 + 2.0 * u[nb:],
    }


def bose_params(K: int, N: int, seed: int) -> dict:
    """Number-conserving bosons on K modes with N particles.

    H = sum_{i != j} c_ij a_i^dag a_j + sum_i U_i n_i^2,  c_ji = conj(c_ij),
    |c_ij| ~ U[0,1), arg c_ij ~ U[0, 2 pi), U_i ~ U[0, 2).  The table lists c_ij
    for i < j in (i-major, j-minor) order.
    """
    npair = K * (K - 1) // 2
    u = uniform(seed, 2 * npair + K)
    mag = u[:npair]
    theta = 2.0 * np.pi * u[npair: 2 * npair]
    return {
        "model": "bose", "K": K, "N": N,
        "c_re": mag * np.cos(theta), "c_im": mag * np.sin(theta),
        "U": 2.0 * u[2 * npair:],
    }


def neel_index(L: int) -> int:
    """Basis index of the Neel state (spin i up for even i, down for odd i)."""
    return sum(1 << i for i in range(1, L, 2))


def bose_dim(K: int, N: int) -> int:
    """Number of occupation tuples of K modes holding N bosons, C(N+K-1, N)."""
    return math.comb(N + K - 1, N)


# ---------------------------------------------------------------- workloads

def workload(name: str) -> dict:
    """Named synthetic workloads (parameters, initial state and solve settings)."""
    if name == "tfim_L12":
        p = tfim_params(12, seed=1)
        return {"name": name, "params": p, "d": 1 << 12, "v0": ("random", 101),
                "t": 10.0, "m": 40, "tol": 1e-8}
    if name == "xxzdm_L22":
        p = xxzdm_params(22, seed=2)
        return {"name": name, "params": p, "d": 1 << 22, "v0": ("index", neel_index(22)),
                "t": 50.0, "m": 40, "tol": 1e-8}
    if name == "xxzdm_L20":
        p = xxzdm_params(20, seed=3)
        return {"name": name, "params": p, "d": 1 << 20, "v0": ("random", 301),
                "t": 50.0, "m": 40, "tol": 1e-8}
    if name == "bose_K14_N10":
        p = bose_params(14, 10, seed=4)
        occ = tuple([1] * 10 + [0] * 4)
        return {"name": name, "params": p, "d": bose_dim(14, 10), "v0": ("occupation", occ),
                "t": 20.0, "m": 50, "tol": 1e-10}
    if name == "random_L20":
        # a general complex128 Hermitian matrix given as COO (one distinct value per
        # coupled pair: ~5.2M values, far above the 65,535 the value-indexed copy takes)
        return {"name": name, "params": {"model": "coo", "L": 20, "seed": 9}, "d": 1 << 20,
                "v0": ("random", 309), "t": 50.0, "m": 40, "tol": 1e-8}
    if name == "batch_xxzdm_L20_x64":
        # 64 random initial vectors under the Hamiltonian of xxzdm_L20
        p = xxzdm_params(20, seed=3)
        return {"name": name, "params": p, "d": 1 << 20, "nvec": 64,
                "v0_seeds": list(range(301, 365)), "t": 50.0, "m": 40, "tol": 1e-8}
    if name == "tfim_multi_x32":
        # 32 independent open TFIM chains: L uniform on 10..20, t ~ U[1, 20]
        u = uniform(6, 64)
        probs = []
        for i in range(32):
            L = 10 + min(int(u[2 * i] * 11), 10)
            probs.append({"params": tfim_params(L, seed=800 + i), "d": 1 << L,
                          "t": float(1.0 + 19.0 * u[2 * i + 1]), "v0_seed": 900 + i})
        return {"name": name, "problems": probs, "m": 30, "tol": 1e-8}
    if name == "memory_scaling":
        # the sizes of the paper's runtime study (Sec. 5): K = K' = 4, 6, 8, 10, Nm = K / 2,
        # N0 = Nc = 100, t = 10, and the memory-limit point K = K' = 10, N0 = Nc = 139
        sizes = [(K, 100) for K in (4, 6, 8, 10)] + [(10, 139)]
        probs = []
        for K, N0 in sizes:
            p = memory_params(K=K, Kp=K, N0=N0, Nm=K // 2, Nc=float(N0))
            probs.append({"params": p, "d": memory_dim(p),
                          "v0": ("occupation", memory_initial_occupation(p))})
        return {"name": name, "sizes": probs, "t": 10.0, "m": 40, "tol": 1e-7}
    if name == "memory_K10_sampled":
        # the same solve with every mode occupation at 100 evenly spaced times
        w = workload("memory_K10")
        w["name"] = name
        w["samples"] = [float(x) for x in np.linspace(0.0, w["t"], 100)]
        return w
    if name == "memory_K10":
        p = memory_params(K=10, Kp=10, N0=100, Nm=5, Nc=100.0)
        return {"name": name, "params": p, "d": memory_dim(p),
                "v0": ("occupation", memory_initial_occupation(p)),
                "t": 10.0, "m": 40, "tol": 1e-7}
    raise KeyError(name)


def initial_block(seeds, d: int) -> np.ndarray:
    """len(seeds) x d block of normalised random states, one row per seed."""
    return np.stack([random_state(s, d) for s in seeds])


def random_hermitian_coo(L: int, seed: int):
    """COO triplets (rows, cols, vals) of a random complex Hermitian matrix of
    dimension 2^L with the sparsity pattern of a periodic spin-1/2 chain with
    nearest-neighbour flip-flop terms: entry (r, r ^ (1 << b | 1 << b+1)) for every
    bond b whose two bits in r differ, and the diagonal.  Every off-diagonal pair
    draws its own value (so there are as many distinct values as pairs):
    H[lo, hi] = 1/2 (1 + u) e^{2 pi i v} for the pair lo < hi on bond b, with u, v
    the uniforms number 2 (lo L + b) and 2 (lo L + b) + 1 of stream ``seed``, and
    H[hi, lo] = conj(H[lo, hi]); the diagonal entries are U[-1, 1) (stream
    seed + 1).  Rows come out unsorted; duplicates do not occur."""
    d = 1 << L
    r = np.arange(d, dtype=np.int64)
    rows, cols, vals = [r], [r], [(2.0 * uniform(seed + 1, d) - 1.0).astype(np.complex128)]
    for b in range(L):
        c = (b + 1) % L
        flip = ((r >> b) & 1) != ((r >> c) & 1)
        src = r[flip]
        dst = src ^ ((1 << b) | (1 << c))
        lo = np.minimum(src, dst)
        key = (lo * L + b).astype(np.uint64)
        u = (splitmix64_at(seed, 2 * key) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        v = (splitmix64_at(seed, 2 * key + 1) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        mag = 0.5 * (1.0 + u)
        val = np.empty(src.size, dtype=np.complex128)
        val.real = mag * np.cos(2.0 * np.pi * v)
        val.imag = mag * np.sin(2.0 * np.pi * v)
        val = np.where(src == lo, val, np.conj(val))
        rows.append(src)
        cols.append(dst)
        vals.append(val)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def initial_vector(spec, d: int, index_of=None) -> np.ndarray:
    """Build the initial vector from a workload's ``v0`` spec.

    ``index_of`` maps an occupation tuple to a basis index; it is supplied by the
    caller (each side uses its own basis ordering).
    """
    kind, arg = spec
    if kind == "random":
        return random_state(arg, d)
    if kind == "index":
        return basis_state(d, arg)
    if kind == "occupation":
        if index_of is None:
            raise ValueError("occupation initial state needs an index_of callable")
        return basis_state(d, int(index_of(arg)))
    raise ValueError(kind)


# ---------------------------------------------------------------- serving mix

SERVE_POOL_SIZE = 16          # Hamiltonians per family in the serving mix
SERVE_BOSE_SHAPES = ((12, 6), (14, 6), (14, 7), (14, 8), (14, 9), (14, 10))


def serve_pool() -> list:
    """The Hamiltonians a serving stream draws from: two families of 16.

    spin: TFIM (even slots) and XXZ-DM (odd slots) chains with L spread evenly
    over 10..22 (2^10..2^22 states); bose: number-conserving bosons cycling over
    (K, N) = (12, 6), (14, 6), (14, 7), (14, 8), (14, 9), (14, 10), i.e.
    12,376..1,144,066 states.  Entries are (family, parameters)."""
    pool = []
    for i in range(SERVE_POOL_SIZE):
        L = 10 + int(round(12 * i / (SERVE_POOL_SIZE - 1)))
        if i % 2 == 0:
            pool.append(("spin", tfim_params(L, seed=500 + i)))
        else:
            pool.append(("spin", xxzdm_params(L, seed=500 + i)))
    for i in range(SERVE_POOL_SIZE):
        K, N = SERVE_BOSE_SHAPES[i % len(SERVE_BOSE_SHAPES)]
        pool.append(("bose", bose_params(K, N, seed=520 + i)))
    return pool


def serve_requests(n: int, seed: int = 5) -> list:
    """n requests: (pool index, t, tol, v0 seed, unit-rate exponential gap).

    Half spin, half bosons (one uniform draw picks the family, the next the
    Hamiltonian within it), t ~ log-uniform on [1, 100], tol uniform over
    {1e-6, 1e-8, 1e-10}; the gap is an Exp(1) draw that the caller divides by
    the arrival rate.  The draws are counter-based, so the first k requests of
    any n are the same."""
    u = uniform(seed, 5 * n)
    out = []
    for i in range(n):
        fam = 0 if u[5 * i] < 0.5 else 1
        k = fam * SERVE_POOL_SIZE + min(int(u[5 * i + 1] * SERVE_POOL_SIZE), SERVE_POOL_SIZE - 1)
        t = float(10.0 ** (2.0 * u[5 * i + 2]))
        tol = (1e-6, 1e-8, 1e-10)[min(int(u[5 * i + 3] * 3), 2)]
        gap = float(-np.log1p(-u[5 * i + 4]))
        out.append((k, t, tol, 700 + i, gap))
    return out


# ---------------------------------------------------------------- the paper's example system

def memory_params(K: int = 4, Kp: int = 4, N0: int = 20, Nm: int = 2, Nc: float = 20.0,
                  dNc: float = 12.0, em: float | None = None, C0: float = 1.0,
                  Cm: float = 1.0) -> dict:
    """Parameters of the paper's example Hamiltonian (Sec. 5, "memory burden" system).

    Two bosonic modes a_0, b_0 holding N0 particles, K + Kp qubit modes holding Nm
    excitations.  Defaults are the paper's default parameter set (eps_m = sqrt(20),
    N0 = Nc = 20, dNc = 12, K = K' = 4, C0 = Cm = 1, Nm = 2).  The coupling of qubits
    p < q (global numbering 1..K+Kp, the second sector after the first) is
    f = F - 1 if F < 0.5 else F with F = (sqrt(2) (p+1)^3 + sqrt(7) (q+1)^5) mod 1,
    which is the paper's f_1, f_2 and f_3 with their index offsets; the table lists
    f for p < q in (p-major, q-minor) order.
    """
    Q = K + Kp
    fs = []
    for p in range(1, Q + 1):
        for q in range(p + 1, Q + 1):
            F = np.mod(np.sqrt(2.0) * (p + 1) ** 3 + np.sqrt(7.0) * (q + 1) ** 5, 1.0)
            fs.append(F - 1.0 if F < 0.5 else F)
    return {"model": "memory", "K": K, "Kp": Kp, "N0": N0, "Nm": Nm, "Nc": float(Nc),
            "dNc": float(dNc), "em": float(np.sqrt(20.0) if em is None else em),
            "C0": float(C0), "Cm": float(Cm), "f": np.array(fs, dtype=np.float64)}


def memory_dim(p: dict) -> int:
    """(N0 + 1) C(K + K', Nm) states: both sectors conserve their occupation."""
    return (p["N0"] + 1) * math.comb(p["K"] + p["Kp"], p["Nm"])


def memory_initial_occupation(p: dict) -> tuple:
    """|N0, 0, 1 x Nm, 0, ...>: all bosons in a_0, the first Nm qubits excited."""
    Q = p["K"] + p["Kp"]
    return (p["N0"], 0) + tuple([1] * p["Nm"] + [0] * (Q - p["Nm"]))
