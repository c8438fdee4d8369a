"""The oracle's one piece of C: the threaded CSR product of csrmv.c (TEST
INFRASTRUCTURE; only tests/, __graft_entry__ and bench.py reach it through the
oracle).

build() compiles csrmv.c with gcc and OpenMP into oracle/_csrmv.so (no FMA
contraction, so x86 and Arm give the same bits); available() says whether it is
there.  ThreadedCSR wraps a scipy CSR matrix so that ``A @ x`` runs the C
product on a given number of threads: the plain definition of the product,
bitwise the same for any thread count (each row is summed by one thread in
storage order).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrmv.c")
LIB = os.path.join(HERE, "_csrmv.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile _csrmv.so if it is missing or older than csrmv.c."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           SRC, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"gcc failed on csrmv.c:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = C.CDLL(LIB)
        lib.oracle_csrmv.restype = None
        lib.oracle_csrmv.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_void_p, C.c_int]
        _lib = lib
    return _lib


def available() -> bool:
    try:
        _load()
        return True
    except Exception:
        return False


class ThreadedCSR:
    """A scipy CSR matrix whose products run on `threads` CPU threads (csrmv.c)."""

    def __init__(self, A, threads: int):
        import scipy.sparse
        A = scipy.sparse.csr_matrix(A)
        self.A = A
        self.shape = A.shape
        self.threads = int(threads)
        self.rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(A.data, dtype=np.complex128)
        self.lib = _load()

    def matvec(self, x, s: float = 1.0) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty(self.shape[0], dtype=np.complex128)
        self.lib.oracle_csrmv(self.shape[0], self.rowptr.ctypes.data, self.col.ctypes.data,
                              self.val.ctypes.data, x.ctypes.data, float(s), y.ctypes.data,
                              self.threads)
        return y

    def __matmul__(self, x):
        return self.matvec(x)
