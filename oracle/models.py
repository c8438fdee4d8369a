"""Oracle Hamiltonian builders for the synthetic workloads (test infrastructure only).

Sec. 3 of the paper builds H from an operator expression: apply the operator to
every basis state and store each resulting coefficient, with the map from a state
to its index held in a hash table (Sec. 4).  The workloads are spin chains and
number-conserving bosons; their parameters come from the ``workloads`` module.

Matrix convention (the standard one): H[i, j] = <i|H|j>, stored as CSR with
ascending columns in every row and the diagonal always stored.  Values are built
with single roundings in a fixed order so that an independent implementation
following the same definitions reproduces them bit for bit:

* spin chains: sigma^z_i = 1 - 2 bit_i(state);
* TFIM diagonal: acc = 0; for bonds b = 0..L-2: acc += -J_b s_b s_{b+1};
  off-diagonal at state ^ (1 << i): -h_i;
* XXZ-DM diagonal: acc = 0; for bonds b: acc += (delta / 4) s_b s_{b+1}; then for
  sites i: acc += (hz_i / 2) s_i.  Bond b joins sites b and (b+1) mod L.  A row
  whose bond b has spin b up and spin b+1 down gets (hop_b / 2) at the state with
  both flipped; the reverse configuration gets conj(hop_b) / 2;
* bosons: basis = occupation tuples (n_0..n_{K-1}) summing to N, in descending
  lexicographic order starting at (N, 0, ..., 0); the row of state n' holds
  sum_i U_i (n'_i)^2 on the diagonal (accumulated in mode order) and, for every
  ordered pair i != j with n'_i >= 1, the entry c_ij sqrt(n'_i) sqrt(n'_j + 1)
  at the column of n' - e_i + e_j (c_ji = conj(c_ij)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse


@dataclass
class CSR:
    d: int
    rowptr: np.ndarray   # int64, d + 1
    col: np.ndarray      # int64, nnz
    val: np.ndarray      # complex128, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        return scipy.sparse.csr_matrix((self.val, self.col, self.rowptr), shape=(self.d, self.d))

    def row(self, r: int):
        b, e = int(self.rowptr[r]), int(self.rowptr[r + 1])
        return self.col[b:e], self.val[b:e]


def coo_to_csr(d: int, rows, cols, vals) -> CSR:
    """COO triplets to CSR: order by (row, col) keeping input order among equal
    keys, then add duplicates left to right in that order.  Explicit zeros stay."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.complex128)
    order = np.lexsort((cols, rows))                  # stable: ties keep input order
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size:
        new = np.ones(rows.size, dtype=bool)
        new[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
        seg = np.cumsum(new) - 1
        out_val = np.zeros(int(seg[-1]) + 1, dtype=np.complex128)
        np.add.at(out_val, seg, vals)                 # unbuffered, in index order
        out_row, out_col = rows[new], cols[new]
    else:
        out_val = np.zeros(0, dtype=np.complex128)
        out_row = out_col = np.zeros(0, dtype=np.int64)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.add.at(rowptr, out_row + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(d, rowptr, out_col, out_val)


def _sz_signs(L: int, r: np.ndarray):
    return [1.0 - 2.0 * ((r >> i) & 1).astype(np.float64) for i in range(L)]


def tfim_csr(p: dict) -> CSR:
    """Transverse-field Ising chain with open boundary (see module docstring)."""
    L = p["L"]
    J, hx = p["J"], p["h"]
    d = 1 << L
    r = np.arange(d, dtype=np.int64)
    s = _sz_signs(L, r)
    diag = np.zeros(d)
    for b in range(L - 1):
        diag = diag + (-J[b]) * (s[b] * s[b + 1])
    rows = [r]
    cols = [r]
    vals = [diag.astype(np.complex128)]
    for i in range(L):
        rows.append(r)
        cols.append(r ^ (1 << i))
        vals.append(np.full(d, -hx[i], dtype=np.complex128))
    return coo_to_csr(d, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def xxzdm_csr(p: dict) -> CSR:
    """XXZ chain with Dzyaloshinskii-Moriya phases (see module docstring)."""
    L, pbc, delta = p["L"], p["pbc"], p["delta"]
    hop_re, hop_im, hz = p["hop_re"], p["hop_im"], p["hz"]
    if pbc and L < 3:
        raise ValueError("periodic XXZ chain needs L >= 3")
    nb = L if pbc else L - 1
    d = 1 << L
    r = np.arange(d, dtype=np.int64)
    s = _sz_signs(L, r)
    diag = np.zeros(d)
    for b in range(nb):
        diag = diag + (delta * 0.25) * (s[b] * s[(b + 1) % L])
    for i in range(L):
        diag = diag + (hz[i] * 0.5) * s[i]
    rows = [r]
    cols = [r]
    vals = [diag.astype(np.complex128)]
    for b in range(nb):
        a, c = b, (b + 1) % L
        bit_a = (r >> a) & 1
        bit_c = (r >> c) & 1
        mask = (1 << a) | (1 << c)
        up_down = (bit_a == 0) & (bit_c == 1)        # spin a up, spin a+1 down
        down_up = (bit_a == 1) & (bit_c == 0)
        ra = r[up_down]
        rows.append(ra)
        cols.append(ra ^ mask)
        vals.append(np.full(ra.size, complex(0.5 * hop_re[b], 0.5 * hop_im[b])))
        rb = r[down_up]
        rows.append(rb)
        cols.append(rb ^ mask)
        vals.append(np.full(rb.size, complex(0.5 * hop_re[b], -(0.5 * hop_im[b]))))
    return coo_to_csr(d, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


# ---------------------------------------------------------------- bosons

def bose_basis(K: int, N: int):
    """All occupation tuples of K modes with N bosons, descending lexicographic."""
    out = []
    cur = [0] * K

    def rec(pos: int, rem: int):
        if pos == K - 1:
            cur[pos] = rem
            out.append(tuple(cur))
            return
        for a in range(rem, -1, -1):
            cur[pos] = a
            rec(pos + 1, rem - a)

    rec(0, N)
    return out


class BoseBasis:
    """Basis list plus the hash table state -> index (Sec. 3, eq. findIndices; Sec. 4)."""

    def __init__(self, K: int, N: int):
        self.K, self.N = K, N
        self.states = bose_basis(K, N)
        self.index = {s: i for i, s in enumerate(self.states)}

    def __len__(self):
        return len(self.states)


def _pair(K: int, i: int, j: int) -> int:
    """Position of c_ij (i < j) in the (i-major, j-minor) table."""
    return i * K - i * (i + 1) // 2 + (j - i - 1)


def bose_row(p: dict, basis: BoseBasis, r: int):
    """Columns (ascending) and values of row r of the bosonic Hamiltonian."""
    K = p["K"]
    c_re, c_im, U = p["c_re"], p["c_im"], p["U"]
    n = basis.states[r]
    acc = 0.0
    for i in range(K):
        acc = acc + U[i] * float(n[i] * n[i])
    entries = [(r, complex(acc, 0.0))]
    for i in range(K):
        if n[i] == 0:
            continue
        for j in range(K):
            if j == i:
                continue
            src = list(n)
            src[i] -= 1
            src[j] += 1
            col = basis.index[tuple(src)]
            amp = math.sqrt(float(n[i])) * math.sqrt(float(n[j] + 1))
            if i < j:
                cr, ci = c_re[_pair(K, i, j)], c_im[_pair(K, i, j)]
            else:
                cr, ci = c_re[_pair(K, j, i)], -c_im[_pair(K, j, i)]
            entries.append((col, complex(cr * amp, ci * amp)))
    entries.sort(key=lambda e: e[0])
    return (np.array([e[0] for e in entries], dtype=np.int64),
            np.array([e[1] for e in entries], dtype=np.complex128))


def bose_csr(p: dict, basis: BoseBasis | None = None) -> CSR:
    """Full bosonic CSR, one row at a time (small K, N only)."""
    basis = basis or BoseBasis(p["K"], p["N"])
    d = len(basis)
    cols, vals, lens = [], [], []
    for r in range(d):
        c, v = bose_row(p, basis, r)
        cols.append(c)
        vals.append(v)
        lens.append(c.size)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    return CSR(d, rowptr, np.concatenate(cols), np.concatenate(vals))


def _desc_rank(keys_desc: np.ndarray, targets: np.ndarray) -> np.ndarray:
    """Positions of `targets` in the strictly decreasing array `keys_desc`
    (every target must be present)."""
    asc = keys_desc[::-1]
    pos = np.searchsorted(asc, targets)
    if not np.all(asc[np.minimum(pos, asc.size - 1)] == targets):
        raise ValueError("target state outside the basis")
    return keys_desc.size - 1 - pos


def _rows_to_csr(d: int, rows, cols, vals) -> CSR:
    """Entries ordered by (row, column); every (row, column) occurs once."""
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1 and np.any((rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])):
        raise ValueError("duplicate entry")
    rowptr = np.zeros(d + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=d))
    return CSR(d, rowptr, cols.astype(np.int64), vals)


def bose_csr_vec(p: dict, basis: BoseBasis | None = None) -> CSR:
    """The matrix of bose_csr, built with array operations over all rows at once.

    For every ordered mode pair (i, j), i != j, each row n with n_i > 0 gets the
    entry sqrt(n_i) sqrt(n_j + 1) c_ij at the rank of n - e_i + e_j (ranks from
    the base-(N+1) key of the occupation tuple, which decreases along the
    descending lexicographic basis); the diagonal is sum_i U_i n_i^2 added in
    mode order.  The roundings are bose_row's, so the two are bitwise equal
    (pinned in tests/test_oracle_models.py)."""
    K, N = p["K"], p["N"]
    basis = basis or BoseBasis(K, N)
    c_re, c_im, U = p["c_re"], p["c_im"], p["U"]
    S = np.array(basis.states, dtype=np.int64)                 # d x K
    d = S.shape[0]
    pw = (N + 1) ** np.arange(K - 1, -1, -1, dtype=np.int64)
    keys = S @ pw
    if d > 1 and not np.all(keys[1:] < keys[:-1]):
        raise ValueError("basis is not in descending lexicographic order")
    r = np.arange(d, dtype=np.int64)
    acc = np.zeros(d)
    for i in range(K):
        acc = acc + U[i] * (S[:, i] * S[:, i]).astype(np.float64)
    rows, cols, vals = [r], [r], [acc.astype(np.complex128)]
    for i in range(K):
        src = S[:, i] > 0
        for j in range(K):
            if j == i:
                continue
            rr = r[src]
            col = _desc_rank(keys, keys[src] + pw[j] - pw[i])
            amp = np.sqrt(S[src, i].astype(np.float64)) * np.sqrt((S[src, j] + 1).astype(np.float64))
            if i < j:
                cr, ci = c_re[_pair(K, i, j)], c_im[_pair(K, i, j)]
            else:
                cr, ci = c_re[_pair(K, j, i)], -c_im[_pair(K, j, i)]
            v = np.empty(rr.size, dtype=np.complex128)
            v.real = cr * amp
            v.imag = ci * amp
            rows.append(rr)
            cols.append(col)
            vals.append(v)
    return _rows_to_csr(d, rows, cols, vals)


def build(p: dict) -> CSR:
    """Dispatch on the parameter table's model name."""
    if p["model"] == "tfim":
        return tfim_csr(p)
    if p["model"] == "xxzdm":
        return xxzdm_csr(p)
    if p["model"] == "bose":
        return bose_csr(p)
    if p["model"] == "memory":
        return memory_csr(p)
    raise ValueError(p["model"])


def spin_row(p: dict, r: int):
    """Row r of a spin-chain Hamiltonian, built entry by entry (for sampled checks
    at sizes where the vectorised builders would be slow)."""
    L = p["L"]
    s = [1.0 - 2.0 * ((r >> i) & 1) for i in range(L)]
    entries = []
    if p["model"] == "tfim":
        acc = 0.0
        for b in range(L - 1):
            acc = acc + (-p["J"][b]) * (s[b] * s[b + 1])
        entries.append((r, complex(acc, 0.0)))
        for i in range(L):
            entries.append((r ^ (1 << i), complex(-p["h"][i], 0.0)))
    elif p["model"] == "xxzdm":
        nb = L if p["pbc"] else L - 1
        acc = 0.0
        for b in range(nb):
            acc = acc + (p["delta"] * 0.25) * (s[b] * s[(b + 1) % L])
        for i in range(L):
            acc = acc + (p["hz"][i] * 0.5) * s[i]
        entries.append((r, complex(acc, 0.0)))
        for b in range(nb):
            a, c = b, (b + 1) % L
            ba, bc = (r >> a) & 1, (r >> c) & 1
            mask = (1 << a) | (1 << c)
            if ba == 0 and bc == 1:
                entries.append((r ^ mask, complex(0.5 * p["hop_re"][b], 0.5 * p["hop_im"][b])))
            elif ba == 1 and bc == 0:
                entries.append((r ^ mask, complex(0.5 * p["hop_re"][b], -(0.5 * p["hop_im"][b]))))
    else:
        raise ValueError(p["model"])
    entries.sort(key=lambda e: e[0])
    return (np.array([e[0] for e in entries], dtype=np.int64),
            np.array([e[1] for e in entries], dtype=np.complex128))


# ---------------------------------------------------------------- the paper's example system

class MemoryBasis:
    """Basis of the paper's example system (Sec. 5): tuples (n0, m0, q_1..q_Q) with
    n0 + m0 = N0 and exactly Nm of the Q = K + K' qubits excited, in descending
    lexicographic order (n0 = N0 first).  Index = (N0 - n0) * C(Q, Nm) + position of
    the qubit tuple among all qubit tuples in descending lexicographic order."""

    def __init__(self, p: dict):
        self.p = p
        Q, Nm = p["K"] + p["Kp"], p["Nm"]
        self.qconf = []
        cur = [0] * Q

        def rec(pos, rem):
            if pos == Q:
                if rem == 0:
                    self.qconf.append(tuple(cur))
                return
            for bit in (1, 0):                         # 1 before 0: descending order
                if bit > rem or Q - pos - 1 < rem - bit:
                    continue
                cur[pos] = bit
                rec(pos + 1, rem - bit)
            cur[pos] = 0

        rec(0, Nm)
        self.qindex = {q: i for i, q in enumerate(self.qconf)}
        self.nq = len(self.qconf)

    def __len__(self):
        return (self.p["N0"] + 1) * self.nq

    def state(self, r: int) -> tuple:
        b, qi = divmod(r, self.nq)
        n0 = self.p["N0"] - b
        return (n0, self.p["N0"] - n0) + self.qconf[qi]

    def index(self, s: tuple) -> int:
        return (self.p["N0"] - s[0]) * self.nq + self.qindex[tuple(s[2:])]


def _qpair(Q: int, p: int, q: int) -> int:
    """Position of f(p, q), p < q (0-based qubits), in the (p-major, q-minor) table."""
    return p * Q - p * (p + 1) // 2 + (q - p - 1)


def memory_row(p: dict, basis: MemoryBasis, r: int):
    """Row r of the example Hamiltonian (Sec. 5, eq. fullHamiltonianSimple):
    C0 (a0^+ b0 + h.c.) + em (1 - n0/Nc) sum_k n_k + em (1 - n0/(Nc - dNc)) sum_k' n'_k'
    + Cm sum_{p<q} f(p,q) (a_p^+ a_q + h.c.) over all qubit pairs.

    Rounding order: diag = (em * (1 - n0 / Nc)) * n1 + (em * (1 - n0 / (Nc - dNc))) * n2;
    boson hops C0 * (sqrt(.) * sqrt(.)); qubit hops Cm * f."""
    K, Q = p["K"], p["K"] + p["Kp"]
    n0, m0 = basis.state(r)[:2]
    qs = basis.state(r)[2:]
    n1, n2 = sum(qs[:K]), sum(qs[K:])
    em, Nc, dNc = p["em"], p["Nc"], p["dNc"]
    diag = (em * (1.0 - n0 / Nc)) * n1 + (em * (1.0 - n0 / (Nc - dNc))) * n2
    entries = [(r, complex(diag, 0.0))]
    if n0 >= 1:       # a0^+ b0 brings (n0 - 1, m0 + 1) to this state
        amp = math.sqrt(float(n0)) * math.sqrt(float(m0 + 1))
        entries.append((basis.index((n0 - 1, m0 + 1) + qs), complex(p["C0"] * amp, 0.0)))
    if m0 >= 1:       # b0^+ a0 brings (n0 + 1, m0 - 1) to this state
        amp = math.sqrt(float(m0)) * math.sqrt(float(n0 + 1))
        entries.append((basis.index((n0 + 1, m0 - 1) + qs), complex(p["C0"] * amp, 0.0)))
    for a in range(Q):
        for b in range(a + 1, Q):
            if qs[a] != qs[b]:
                src = list(qs)
                src[a], src[b] = qs[b], qs[a]
                col = basis.index((n0, m0) + tuple(src))
                entries.append((col, complex(p["Cm"] * p["f"][_qpair(Q, a, b)], 0.0)))
    entries.sort(key=lambda e: e[0])
    return (np.array([e[0] for e in entries], dtype=np.int64),
            np.array([e[1] for e in entries], dtype=np.complex128))


def memory_csr(p: dict, basis: MemoryBasis | None = None) -> CSR:
    basis = basis or MemoryBasis(p)
    d = len(basis)
    cols, vals, lens = [], [], []
    for r in range(d):
        c, v = memory_row(p, basis, r)
        cols.append(c)
        vals.append(v)
        lens.append(c.size)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    return CSR(d, rowptr, np.concatenate(cols), np.concatenate(vals))


def memory_csr_vec(p: dict, basis: MemoryBasis | None = None) -> CSR:
    """The matrix of memory_csr, built with array operations over all rows at once.

    Row (b, q) (n0 = N0 - b, qubit tuple q) holds the diagonal, the two boson
    hops to blocks b + 1 (n0 - 1) and b - 1 (m0 - 1), and one qubit hop per pair
    a < b' with q_a != q_b' to the swapped tuple in the same block.  The qubit
    hops' targets are found once per qubit tuple (the same in every block).  The
    roundings are memory_row's, so the two are bitwise equal (pinned in
    tests/test_oracle_models.py)."""
    basis = basis or MemoryBasis(p)
    K, Q, N0 = p["K"], p["K"] + p["Kp"], p["N0"]
    em, Nc, dNc, C0, Cm = p["em"], p["Nc"], p["dNc"], p["C0"], p["Cm"]
    qc = np.array(basis.qconf, dtype=np.int64)                 # nq x Q
    nq = qc.shape[0]
    d = len(basis)
    pw = 2 ** np.arange(Q - 1, -1, -1, dtype=np.int64)
    qkeys = qc @ pw                                            # decreasing along the basis
    n1 = qc[:, :K].sum(axis=1)
    n2 = qc[:, K:].sum(axis=1)
    hop_src, hop_dst, hop_val = [], [], []
    qi = np.arange(nq, dtype=np.int64)
    for a in range(Q):
        for b2 in range(a + 1, Q):
            diff = qc[:, a] != qc[:, b2]
            tk = qkeys[diff] + (qc[diff, b2] - qc[diff, a]) * pw[a] + (qc[diff, a] - qc[diff, b2]) * pw[b2]
            hop_src.append(qi[diff])
            hop_dst.append(_desc_rank(qkeys, tk))
            hop_val.append(np.full(int(diff.sum()), complex(Cm * p["f"][_qpair(Q, a, b2)], 0.0)))
    hop_src = np.concatenate(hop_src)
    hop_dst = np.concatenate(hop_dst)
    hop_val = np.concatenate(hop_val)
    rows, cols, vals = [], [], []
    for blk in range(N0 + 1):
        n0 = N0 - blk
        m0 = N0 - n0
        base = blk * nq
        diag = (em * (1.0 - n0 / Nc)) * n1.astype(np.float64) + \
               (em * (1.0 - n0 / (Nc - dNc))) * n2.astype(np.float64)
        rows.append(base + qi)
        cols.append(base + qi)
        vals.append(diag.astype(np.complex128))
        if n0 >= 1:
            amp = math.sqrt(float(n0)) * math.sqrt(float(m0 + 1))
            rows.append(base + qi)
            cols.append(base + nq + qi)
            vals.append(np.full(nq, complex(C0 * amp, 0.0)))
        if m0 >= 1:
            amp = math.sqrt(float(m0)) * math.sqrt(float(n0 + 1))
            rows.append(base + qi)
            cols.append(base - nq + qi)
            vals.append(np.full(nq, complex(C0 * amp, 0.0)))
        rows.append(base + hop_src)
        cols.append(base + hop_dst)
        vals.append(hop_val)
    return _rows_to_csr(d, rows, cols, vals)


def memory_norm1(p: dict, basis: MemoryBasis | None = None) -> float:
    """||H||_1 (maximum absolute row sum; H is real symmetric) of the example
    Hamiltonian, vectorised over the basis without assembling H."""
    basis = basis or MemoryBasis(p)
    K, Q, N0 = p["K"], p["K"] + p["Kp"], p["N0"]
    qc = np.array(basis.qconf, dtype=np.int64)                 # nq x Q
    n1 = qc[:, :K].sum(axis=1).astype(np.float64)
    n2 = qc[:, K:].sum(axis=1).astype(np.float64)
    hop = np.zeros(len(qc))
    for a in range(Q):
        for b in range(a + 1, Q):
            hop += (qc[:, a] != qc[:, b]) * abs(p["Cm"] * p["f"][_qpair(Q, a, b)])
    best = 0.0
    for n0 in range(N0 + 1):
        m0 = N0 - n0
        diag = np.abs((p["em"] * (1.0 - n0 / p["Nc"])) * n1
                      + (p["em"] * (1.0 - n0 / (p["Nc"] - p["dNc"]))) * n2)
        bos = 0.0
        if n0 >= 1:
            bos += abs(p["C0"] * math.sqrt(n0) * math.sqrt(m0 + 1))
        if m0 >= 1:
            bos += abs(p["C0"] * math.sqrt(m0) * math.sqrt(n0 + 1))
        best = max(best, float(np.max(diag + hop + bos)))
    return best


# ---------------------------------------------------------------- observables

def occupation(p: dict, l: int) -> np.ndarray:
    """Number operator of mode l as the diagonal over the model's basis (float64).

    Spin chains: mode l is site l and n_l = 1 when spin l points down (bit l of
    the index).  Bosons: the occupation of mode l.  The paper's example system
    (Sec. 5): mode 0 is a_0 (n0), mode 1 is b_0 (m0), modes 2.. are the qubits
    a_1..a_K, a'_1..a'_K' -- the number operators whose expectation values the
    paper plots over time.
    """
    kind = p["model"]
    if kind in ("tfim", "xxzdm"):
        d = 1 << p["L"]
        return ((np.arange(d, dtype=np.int64) >> l) & 1).astype(np.float64)
    if kind == "bose":
        b = BoseBasis(p["K"], p["N"])
        return np.array([s[l] for s in b.states], dtype=np.float64)
    if kind == "memory":
        b = MemoryBasis(p)
        return np.array([b.state(r)[l] for r in range(len(b))], dtype=np.float64)
    raise KeyError(kind)


# ---------------------------------------------------------------- operator expressions (Sec. 3)

def operator_basis(L: int, N: int, caps=None) -> list:
    """All occupation tuples (n_1..n_L) with sum N and n_l <= caps[l] (Sec. 3,
    eq. totalOccupationNumber and the fixed maximal occupations of Sec. 4), in
    descending lexicographic order; ind(state) = position in this list."""
    caps = [N] * L if caps is None else [min(int(c), N) for c in caps]
    out, cur = [], [0] * L

    def rec(pos: int, rem: int):
        if pos == L:
            if rem == 0:
                out.append(tuple(cur))
            return
        for a in range(min(rem, caps[pos]), -1, -1):
            cur[pos] = a
            rec(pos + 1, rem - a)
        cur[pos] = 0

    rec(0, N)
    return out


def apply_term(state: tuple, factors, caps, N: int):
    """Apply one product of ladder operators (listed left to right; the rightmost
    acts first) to a number state: returns (target state, product of the integer
    factors under the square root) or None when the result is zero or leaves
    the space.  a_l |n_l> = sqrt(n_l) |n_l - 1>, a_l^dag |n_l> = sqrt(n_l + 1) |n_l + 1>."""
    occ = list(state)
    prod = 1
    for mode, dag in reversed(factors):
        if dag:
            occ[mode] += 1
            if occ[mode] > caps[mode]:
                return None
            prod *= occ[mode]
        else:
            if occ[mode] == 0:
                return None
            prod *= occ[mode]
            occ[mode] -= 1
    if sum(occ) != N:
        return None
    return tuple(occ), prod


def operator_csr(op: dict) -> CSR:
    """createMatrix (Sec. 3) for a Hermitian operator given as terms.

    op = {"L", "N", "caps" (or None), "terms": [(coef complex, [(mode, dagger), ...]), ...]}.
    Row j holds <j|H|i> for the states i reached from state j: applying the
    operator to |j> gives sum_k c_k |i_k>, i.e. <i_k|H|j> = c_k, and for a
    Hermitian operator <j|H|i_k> = conj(c_k).  Contributions to the same column
    are added in term order; every diagonal entry is stored.
    """
    L, N = op["L"], op["N"]
    caps = [N] * L if op.get("caps") is None else [min(int(c), N) for c in op["caps"]]
    states = operator_basis(L, N, caps)
    index = {s: i for i, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for j, s in enumerate(states):
        acc = {j: 0j}
        for coef, factors in op["terms"]:
            r = apply_term(s, factors, caps, N)
            if r is None:
                continue
            tgt, prod = r
            i = index[tgt]
            v = complex(coef).conjugate() * np.sqrt(float(prod))
            acc[i] = acc.get(i, 0j) + v
        for i in sorted(acc):
            rows.append(j)
            cols.append(i)
            vals.append(acc[i])
    d = len(states)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.add.at(rowptr, np.asarray(rows, dtype=np.int64) + 1, 1)
    return CSR(d, np.cumsum(rowptr), np.asarray(cols, dtype=np.int64),
               np.asarray(vals, dtype=np.complex128))
