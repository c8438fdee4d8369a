"""Python binding of libte (ctypes): argument marshalling only.

Every function mirrors the C entry point of the same name in ``include/te.h``;
all arithmetic happens in libte's CUDA kernels.  Vectors are numpy complex128
arrays (host) or torch complex128 CUDA tensors (device); the binding sets
TE_PTR_DEVICE accordingly.  Loading fails loudly when libte.so is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libte.so")

TE_OK = 0
TE_PENDING = 1
TE_ERR_INVALID_ARG = -1
TE_ERR_CUDA = -2
TE_ERR_OOM = -3
TE_ERR_NOT_HERMITIAN = -4
TE_ERR_NOT_NORMALIZED = -5
TE_ERR_STEP_UNDERFLOW = -6
TE_ERR_NONFINITE = -7
TE_ERR_TIMEOUT = -8
TE_ERR_CANCELLED = -9
TE_ERR_UNSUPPORTED = -10
TE_ERR_INTERNAL = -11

TE_PTR_DEVICE = 0x1
TE_CHECK_HERMITIAN = 0x2
TE_INPUT_IS_CSR = 0x4
TE_WARN_ROUNDOFF = 0x1
TE_WARN_QUAD = 0x2
TE_FLAG_BREAKDOWN = 0x4
TE_M_MAX = 128
TE_NOALLOC_MAX_D = 8388608
TE_BATCH_MAX = 64
TE_MULTI_MAX = 256
TE_QUAD_TANH_SINH = 0
TE_QUAD_GAUSS = 1
TE_REORTH_NONE = 0
TE_REORTH_FULL = 1
TE_OPT_PROFILE = 0x10
TE_OPT_TEST_FUSED_TIMEOUT = 0x20
TE_FLAG_FUSED_RETRY = 0x8
TE_SMALLEXP_CHEB = 0
TE_SMALLEXP_EIG = 1
TE_FUSED_AUTO = 0
TE_FUSED_OFF = 1
TE_MODEL_TFIM = 1
TE_MODEL_XXZDM = 2
TE_MODEL_BOSE = 3
TE_MODEL_MEMORY = 4
TE_SERVE_BATCH = 0
TE_SERVE_SOLO = 1


class te_options(C.Structure):
    _fields_ = [("quad", C.c_int32), ("gauss_n", C.c_int32), ("n_substeps", C.c_int32),
                ("reorth", C.c_int32), ("t_step0", C.c_double), ("shrink", C.c_double),
                ("quad_rel_tol", C.c_double), ("quad_max_levels", C.c_int32),
                ("max_substeps", C.c_int32), ("min_step_rel", C.c_double), ("flags", C.c_uint32),
                ("spmv_lanes", C.c_int32), ("small_exp", C.c_int32), ("fused_lanczos", C.c_int32)]


class te_stats(C.Structure):
    _fields_ = [("restarts", C.c_int64), ("matvecs", C.c_int64), ("breakdowns", C.c_int64),
                ("quad_warnings", C.c_int64), ("err_bound", C.c_double),
                ("roundoff_est", C.c_double), ("t_reached", C.c_double), ("norm_in", C.c_double),
                ("flags", C.c_uint32), ("m_used", C.c_int32), ("spmv_ms", C.c_double),
                ("spmv_launches", C.c_int64), ("solve_ms", C.c_double),
                ("quad_integrals", C.c_int64), ("quad_nodes", C.c_int64),
                ("eig_mcycles", C.c_double), ("search_mcycles", C.c_double),
                ("fused_restarts", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class te_matrix_info(C.Structure):
    _fields_ = [("d", C.c_int64), ("nnz", C.c_int64), ("norm1", C.c_double),
                ("max_row_nnz", C.c_int32), ("spmv_lanes", C.c_int32), ("sell_nnz", C.c_int64),
                ("sell_dict", C.c_int32), ("sell_tpt", C.c_int32),
                ("sell_real", C.c_int32), ("sell_async", C.c_int32)]


class te_model_desc(C.Structure):
    _fields_ = [("model", C.c_int32), ("L", C.c_int32), ("N", C.c_int32), ("pbc", C.c_int32),
                ("delta", C.c_double), ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("c", C.POINTER(C.c_double)), ("L2", C.c_int32), ("N2", C.c_int32),
                ("p", C.POINTER(C.c_double))]


class te_operator_desc(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("n_particles", C.c_int32),
                ("max_occ", C.POINTER(C.c_int32)), ("n_terms", C.c_int32),
                ("term_len", C.POINTER(C.c_int32)), ("modes", C.POINTER(C.c_int32)),
                ("dagger", C.POINTER(C.c_int32)), ("coef", C.POINTER(C.c_double))]


# te_allocator's callbacks (include/te.h)
TE_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32, C.c_void_p)
TE_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p)


class te_allocator(C.Structure):
    _fields_ = [("alloc", TE_ALLOC_FN), ("free", TE_FREE_FN), ("user", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "te_version": (C.c_char_p, []),
    "te_status_string": (C.c_char_p, [C.c_int32]),
    "te_default_options": (None, [C.POINTER(te_options)]),
    "te_create": (C.c_int32, [C.POINTER(_P), C.c_int32, _P]),
    "te_create_with_allocator": (C.c_int32, [C.POINTER(_P), C.c_int32, _P, C.POINTER(te_allocator)]),
    "te_destroy": (None, [_P]),
    "te_last_error": (C.c_char_p, [_P]),
    "te_build_csr": (C.c_int32, [_P, C.c_int64, C.c_int64, _P, _P, _P, C.c_uint32, C.POINTER(_P)]),
    "te_build_model": (C.c_int32, [_P, C.POINTER(te_model_desc), C.POINTER(_P)]),
    "te_model_basis_index": (C.c_int32, [C.POINTER(te_model_desc), _P, C.POINTER(C.c_int64)]),
    "te_matrix_info_get": (C.c_int32, [_P, C.POINTER(te_matrix_info)]),
    "te_matrix_export": (C.c_int32, [_P, _P, _P, _P, _P, C.c_uint32]),
    "te_matrix_free": (None, [_P]),
    "te_matrix_tune": (C.c_int32, [_P, _P, C.c_int32, C.POINTER(C.c_double)]),
    "te_measure_fp64": (C.c_int32, [_P, C.POINTER(C.c_double)]),
    "te_measure_fp64_mma": (C.c_int32, [_P, C.POINTER(C.c_double)]),
    "te_matrix_set_sell": (C.c_int32, [_P, _P, C.c_int32, C.c_int32]),
    "te_fused_barrier_check": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_double)]),
    "te_spmv": (C.c_int32, [_P, _P, _P, _P, C.POINTER(C.c_double), C.c_uint32]),
    "te_spmv_noalloc": (C.c_int32, [_P, _P, _P, _P, C.POINTER(C.c_double), C.c_uint32]),
    "te_evolve": (C.c_int32, [_P, _P, _P, C.c_double, C.c_double, C.c_int32,
                              C.POINTER(te_options), _P, C.POINTER(te_stats)]),
    "te_evolve_sampled": (C.c_int32, [_P, _P, _P, C.c_double, C.c_int32, _P, C.c_double,
                                      C.c_int32, C.POINTER(te_options), _P, _P, C.c_int32, _P,
                                      _P, _P, C.POINTER(te_stats)]),
    "te_build_operator": (C.c_int32, [_P, C.POINTER(te_operator_desc), C.POINTER(_P)]),
    "te_operator_basis_index": (C.c_int32, [C.POINTER(te_operator_desc), _P, C.POINTER(C.c_int64)]),
    "te_operator_occupation": (C.c_int32, [_P, C.POINTER(te_operator_desc), C.c_int32, _P,
                                           C.c_uint32]),
    "te_model_occupation": (C.c_int32, [_P, C.POINTER(te_model_desc), C.c_int32, _P, C.c_uint32]),
    "te_evolve_batch": (C.c_int32, [_P, _P, C.c_int32, _P, C.c_double, C.c_double, C.c_int32,
                                    C.POINTER(te_options), _P, _P, _P]),
    "te_evolve_multi": (C.c_int32, [_P, C.c_int32, _P, _P, _P, C.c_double, C.c_int32,
                                    C.POINTER(te_options), _P, _P, _P]),
    "te_submit": (C.c_int32, [_P, _P, _P, C.c_double, C.c_double, C.c_int32,
                              C.POINTER(te_options), C.POINTER(_P)]),
    "te_poll": (C.c_int32, [_P, _P, C.POINTER(te_stats)]),
    "te_wait": (C.c_int32, [_P, C.c_double, _P, C.POINTER(te_stats)]),
    "te_cancel": (C.c_int32, [_P]),
    "te_request_free": (None, [_P]),
    "te_set_memory_budget": (C.c_int32, [_P, C.c_int64]),
    "te_serve_config": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64]),
}

_lib = None


def lib():
    """Load libte.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libte.so not found at {LIB_PATH}; build it first "
                               "(python -m paper_2205_15346_gb300.build)")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def exported_symbols():
    return sorted(_SIGS)


class TEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{te_status_string(status)}: {msg}")
        self.status = status


def te_status_string(s: int) -> str:
    return lib().te_status_string(s).decode()


def te_version() -> str:
    return lib().te_version().decode()


def _check(ctx, status: int, allow=(TE_OK,)):
    if status not in allow:
        msg = lib().te_last_error(ctx).decode() if ctx else ""
        raise TEError(status, msg)
    return status


# ---------------------------------------------------------------- marshalling helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _vec_ptr(x, d: int, writable: bool = False):
    """(pointer, is_device, keepalive) for a complex128 vector of length d."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.complex128 or x.numel() != d or not x.is_contiguous():
            raise ValueError("expected a contiguous complex128 tensor of length d")
        return C.c_void_p(x.data_ptr()), x.is_cuda, x
    a = np.asarray(x)
    if a.dtype != np.complex128 or a.size != d or not a.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError("output must be a contiguous complex128 array of length d")
        a = np.ascontiguousarray(a, dtype=np.complex128).reshape(-1)
        if a.size != d:
            raise ValueError("vector length does not match d")
    return C.c_void_p(a.ctypes.data), False, a


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(C.POINTER(C.c_double)), a


def te_default_options() -> te_options:
    o = te_options()
    lib().te_default_options(C.byref(o))
    return o


def make_options(**kw) -> te_options:
    o = te_default_options()
    for k, v in kw.items():
        if k == "quad" and isinstance(v, str):
            v = {"tanh-sinh": TE_QUAD_TANH_SINH, "gauss": TE_QUAD_GAUSS}[v]
        if k == "small_exp" and isinstance(v, str):
            v = {"cheb": TE_SMALLEXP_CHEB, "eig": TE_SMALLEXP_EIG}[v]
        if k == "reorth" and isinstance(v, bool):
            v = TE_REORTH_FULL if v else TE_REORTH_NONE
        if k == "profile":
            o.flags |= TE_OPT_PROFILE if v else 0
            continue
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------- C entry points

# callbacks handed to te_create_with_allocator, kept alive until te_destroy
_ALLOCATORS = {}


class TorchAllocator:
    """A te_allocator that takes the library's device memory from PyTorch's
    caching allocator (torch.cuda.caching_allocator_alloc / _delete), so that the
    Krylov bases and matrices share the pool torch.cuda.memory_allocated reports.
    The blocks are allocated on the context's stream, which the library
    synchronises before it frees them."""

    def __init__(self):
        import torch
        self._torch = torch
        self.live = {}                        # pointer -> bytes

        def _alloc(user, nbytes, device, stream):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), int(device), int(stream or 0))
            except Exception:
                return None
            self.live[int(ptr)] = int(nbytes)
            return int(ptr)

        def _free(user, ptr, device, stream):
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._afn = TE_ALLOC_FN(_alloc)
        self._ffn = TE_FREE_FN(_free)
        self.struct = te_allocator(self._afn, self._ffn, None)

    def bytes_live(self) -> int:
        return sum(self.live.values())


def te_create(device: int = 0, stream=None, allocator=None):
    """Context on ``device``; ``stream`` is a cudaStream_t handle (int) or None
    (then torch's current stream on that device, if torch is loaded).
    ``allocator``: None (cudaMalloc) or an object with a ``struct`` attribute
    holding a te_allocator (e.g. TorchAllocator()); it is kept alive until
    te_destroy."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream(device).cuda_stream
        except Exception:
            stream = None
    out = C.c_void_p()
    if allocator is None:
        s = lib().te_create(C.byref(out), device, C.c_void_p(stream or 0))
    else:
        s = lib().te_create_with_allocator(C.byref(out), device, C.c_void_p(stream or 0),
                                           C.byref(allocator.struct))
    _check(None, s)
    if allocator is not None:
        _ALLOCATORS[out.value] = allocator
    return out


def te_destroy(ctx) -> None:
    lib().te_destroy(ctx)
    _ALLOCATORS.pop(ctx.value if isinstance(ctx, C.c_void_p) else ctx, None)


def te_last_error(ctx) -> str:
    return lib().te_last_error(ctx).decode()


def model_desc(params: dict):
    """te_model_desc from a parameter table of the ``workloads`` module (plus keepalives)."""
    m = params["model"]
    desc = te_model_desc()
    keep = []
    if m == "tfim":
        desc.model, desc.L = TE_MODEL_TFIM, params["L"]
        desc.a, k1 = _dptr(params["J"])
        desc.b, k2 = _dptr(params["h"])
        keep = [k1, k2]
    elif m == "xxzdm":
        desc.model, desc.L = TE_MODEL_XXZDM, params["L"]
        desc.pbc, desc.delta = int(params["pbc"]), float(params["delta"])
        desc.a, k1 = _dptr(params["hop_re"])
        desc.b, k2 = _dptr(params["hop_im"])
        desc.c, k3 = _dptr(params["hz"])
        keep = [k1, k2, k3]
    elif m == "bose":
        desc.model, desc.L, desc.N = TE_MODEL_BOSE, params["K"], params["N"]
        desc.a, k1 = _dptr(params["c_re"])
        desc.b, k2 = _dptr(params["c_im"])
        desc.c, k3 = _dptr(params["U"])
        keep = [k1, k2, k3]
    elif m == "memory":
        desc.model, desc.L, desc.L2 = TE_MODEL_MEMORY, params["K"], params["Kp"]
        desc.N, desc.N2 = params["Nm"], params["N0"]
        desc.a, k1 = _dptr(params["f"] if len(params["f"]) else np.zeros(1))
        desc.p, k2 = _dptr([params["Nc"], params["dNc"], params["em"], params["C0"], params["Cm"]])
        keep = [k1, k2]
    else:
        raise ValueError(m)
    return desc, keep


def te_build_model(ctx, params: dict):
    desc, keep = model_desc(params)
    out = C.c_void_p()
    _check(ctx, lib().te_build_model(ctx, C.byref(desc), C.byref(out)))
    return out


def te_model_basis_index(params: dict, occ) -> int:
    desc, keep = model_desc(params)
    o = np.ascontiguousarray(occ, dtype=np.int32)
    idx = C.c_int64()
    _check(None, lib().te_model_basis_index(C.byref(desc), C.c_void_p(o.ctypes.data), C.byref(idx)))
    return idx.value


def te_build_csr(ctx, d: int, rows, cols, vals, flags: int = 0):
    """H from COO (or CSR with TE_INPUT_IS_CSR) host arrays; vals complex128."""
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    v = np.ascontiguousarray(vals, dtype=np.complex128)
    n = c.size
    out = C.c_void_p()
    _check(ctx, lib().te_build_csr(ctx, d, n, C.c_void_p(r.ctypes.data), C.c_void_p(c.ctypes.data),
                                   C.c_void_p(v.ctypes.data), flags, C.byref(out)))
    return out


def te_matrix_info_get(H) -> dict:
    info = te_matrix_info()
    _check(None, lib().te_matrix_info_get(H, C.byref(info)))
    return {name: getattr(info, name) for name, _ in info._fields_}


def te_matrix_export(ctx, H):
    """(rowptr int32, col int32, val complex128) host copies of the CSR arrays."""
    info = te_matrix_info_get(H)
    rp = np.empty(info["d"] + 1, dtype=np.int32)
    col = np.empty(info["nnz"], dtype=np.int32)
    val = np.empty(info["nnz"], dtype=np.complex128)
    _check(ctx, lib().te_matrix_export(ctx, H, C.c_void_p(rp.ctypes.data), C.c_void_p(col.ctypes.data),
                                       C.c_void_p(val.ctypes.data), 0))
    return rp, col, val


def te_matrix_tune(ctx, H, repeats: int = 5) -> float:
    """Autotune H's sliced SpMV on this GPU; returns the best product time (ms)."""
    best = C.c_double()
    _check(ctx, lib().te_matrix_tune(ctx, H, int(repeats), C.byref(best)))
    return best.value


def te_matrix_set_sell(ctx, H, slices_per_task: int, async_trip: int = 0) -> None:
    """Pin the sliced SpMV's work-item size and gather staging (0, 2 or 4)."""
    _check(ctx, lib().te_matrix_set_sell(ctx, H, int(slices_per_task), int(async_trip)))


def te_measure_fp64(ctx) -> float:
    """The FP64 FMA rate this GPU sustains on independent chains (TFLOP/s)."""
    r = C.c_double()
    _check(ctx, lib().te_measure_fp64(ctx, C.byref(r)))
    return r.value


def te_measure_fp64_mma(ctx) -> float:
    """The FP64 rate of the GPU's FP64 matrix instruction (mma.sync m8n8k4, TFLOP/s)."""
    r = C.c_double()
    _check(ctx, lib().te_measure_fp64_mma(ctx, C.byref(r)))
    return r.value


def te_fused_barrier_check(ctx, absent_block: int = -1) -> tuple:
    """One grid barrier of the fused Lanczos loop with block `absent_block`
    missing (-1: none).  Returns (status, blocks that passed, kernel ms); the
    status is TE_ERR_TIMEOUT when the other blocks gave up waiting."""
    n = C.c_int32()
    ms = C.c_double()
    st = _check(ctx, lib().te_fused_barrier_check(ctx, int(absent_block), C.byref(n), C.byref(ms)),
                allow=(TE_OK, TE_ERR_TIMEOUT))
    return st, n.value, ms.value


def te_matrix_free(H) -> None:
    lib().te_matrix_free(H)


def te_spmv(ctx, H, x, y=None):
    """y = H x; returns (y, Re <x, H x>)."""
    d = te_matrix_info_get(H)["d"]
    xp, xdev, xk = _vec_ptr(x, d)
    if y is None:
        if xdev:
            import torch
            y = torch.empty_like(x)
        else:
            y = np.empty(d, dtype=np.complex128)
    yp, ydev, yk = _vec_ptr(y, d, writable=True)
    if xdev != ydev:
        raise ValueError("x and y must both be host or both be device buffers")
    dot = C.c_double()
    _check(ctx, lib().te_spmv(ctx, H, xp, yp, C.byref(dot), TE_PTR_DEVICE if xdev else 0))
    return y, dot.value


def te_spmv_noalloc(ctx, H, x, y):
    """y = H x through the allocation-free entry point; x, y are CUDA tensors.
    Returns Re <x, H x>."""
    d = te_matrix_info_get(H)["d"]
    xp, xdev, xk = _vec_ptr(x, d)
    yp, ydev, yk = _vec_ptr(y, d, writable=True)
    dot = C.c_double()
    flags = TE_PTR_DEVICE if (xdev and ydev) else 0
    _check(ctx, lib().te_spmv_noalloc(ctx, H, xp, yp, C.byref(dot), flags))
    return dot.value


def te_evolve(ctx, H, v_in, t: float, tol: float, m: int, opt: te_options | None = None,
              v_out=None, allow=(TE_OK,)):
    """exp(-iHt) v_in; returns (v_out, stats dict, status)."""
    d = te_matrix_info_get(H)["d"]
    ip, idev, ik = _vec_ptr(v_in, d)
    if v_out is None:
        if idev:
            import torch
            v_out = torch.empty_like(v_in)
        else:
            v_out = np.empty(d, dtype=np.complex128)
    op, odev, ok = _vec_ptr(v_out, d, writable=True)
    if idev != odev:
        raise ValueError("v_in and v_out must both be host or both be device buffers")
    o = opt if opt is not None else te_default_options()
    o = te_options.from_buffer_copy(o)
    o.flags = (o.flags & ~TE_PTR_DEVICE) | (TE_PTR_DEVICE if idev else 0)
    st = te_stats()
    s = lib().te_evolve(ctx, H, ip, float(t), float(tol), int(m), C.byref(o), op, C.byref(st))
    _check(ctx, s, allow)
    return v_out, st.as_dict(), s


def _block_ptr(x, nvec: int, d: int, writable: bool = False):
    """(pointer, is_device, keepalive) for nvec complex128 vectors of length d, one after another."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.complex128 or x.numel() != nvec * d or not x.is_contiguous():
            raise ValueError("expected a contiguous complex128 tensor of nvec x d elements")
        return C.c_void_p(x.data_ptr()), x.is_cuda, x
    a = np.asarray(x)
    if a.dtype != np.complex128 or a.size != nvec * d or not a.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError("output must be a contiguous complex128 array of nvec x d elements")
        a = np.ascontiguousarray(a, dtype=np.complex128).reshape(-1)
        if a.size != nvec * d:
            raise ValueError("block size does not match nvec x d")
    return C.c_void_p(a.ctypes.data), False, a


def te_evolve_batch(ctx, H, v_in, t: float, tol: float, m: int, opt: te_options | None = None,
                    v_out=None, allow=(TE_OK,)):
    """exp(-iHt) applied to every row of v_in (shape (nvec, d)); returns
    (v_out, list of stats dicts, list of per-vector statuses, call status)."""
    d = te_matrix_info_get(H)["d"]
    nvec = int(v_in.shape[0])
    ip, idev, ik = _block_ptr(v_in, nvec, d)
    if v_out is None:
        if idev:
            import torch
            v_out = torch.empty_like(v_in)
        else:
            v_out = np.empty((nvec, d), dtype=np.complex128)
    op, odev, ok = _block_ptr(v_out, nvec, d, writable=True)
    if idev != odev:
        raise ValueError("v_in and v_out must both be host or both be device buffers")
    o = te_options.from_buffer_copy(opt if opt is not None else te_default_options())
    o.flags = (o.flags & ~TE_PTR_DEVICE) | (TE_PTR_DEVICE if idev else 0)
    sts = (te_stats * nvec)()
    stat = (C.c_int32 * nvec)()
    s = lib().te_evolve_batch(ctx, H, nvec, ip, float(t), float(tol), int(m), C.byref(o), op,
                              C.cast(sts, C.c_void_p), C.cast(stat, C.c_void_p))
    _check(ctx, s, allow)
    return v_out, [x.as_dict() for x in sts], [int(x) for x in stat], s


def te_evolve_multi(ctx, Hs, v_ins, ts, tol: float, m: int, opt: te_options | None = None,
                    v_outs=None, allow=(TE_OK,)):
    """Independent solves exp(-i H_i t_i) v_i advanced together; returns
    (list of outputs, list of stats dicts, list of per-problem statuses, call status)."""
    n = len(Hs)
    if len(v_ins) != n or len(ts) != n:
        raise ValueError("Hs, v_ins and ts must have the same length")
    ds = [te_matrix_info_get(H)["d"] for H in Hs]
    ins = [_vec_ptr(v, d) for v, d in zip(v_ins, ds)]
    dev = ins[0][1]
    if any(x[1] != dev for x in ins):
        raise ValueError("all vectors must be host arrays or all device tensors")
    if v_outs is None:
        if dev:
            import torch
            v_outs = [torch.empty_like(v) for v in v_ins]
        else:
            v_outs = [np.empty(d, dtype=np.complex128) for d in ds]
    outs = [_vec_ptr(v, d, writable=True) for v, d in zip(v_outs, ds)]
    if any(x[1] != dev for x in outs):
        raise ValueError("outputs must live where the inputs do")
    o = te_options.from_buffer_copy(opt if opt is not None else te_default_options())
    o.flags = (o.flags & ~TE_PTR_DEVICE) | (TE_PTR_DEVICE if dev else 0)
    Harr = (C.c_void_p * n)(*[C.c_void_p(H.value if isinstance(H, C.c_void_p) else H) for H in Hs])
    inarr = (C.c_void_p * n)(*[x[0] for x in ins])
    outarr = (C.c_void_p * n)(*[x[0] for x in outs])
    tarr = (C.c_double * n)(*[float(x) for x in ts])
    sts = (te_stats * n)()
    stat = (C.c_int32 * n)()
    s = lib().te_evolve_multi(ctx, n, C.cast(Harr, C.c_void_p), C.cast(inarr, C.c_void_p),
                              C.cast(tarr, C.c_void_p), float(tol), int(m), C.byref(o),
                              C.cast(outarr, C.c_void_p), C.cast(sts, C.c_void_p),
                              C.cast(stat, C.c_void_p))
    _check(ctx, s, allow)
    return v_outs, [x.as_dict() for x in sts], [int(x) for x in stat], s


def operator_desc(op: dict):
    """te_operator_desc for {"L", "N", "caps" (or None), "terms": [(coef, [(mode, dagger), ...])]}
    (the oracle's format); returns (desc, keepalive)."""
    L, N = int(op["L"]), int(op["N"])
    terms = op["terms"]
    tl = np.array([len(f) for _, f in terms], dtype=np.int32)
    modes = np.array([m for _, f in terms for (m, _) in f] or [0], dtype=np.int32)
    dag = np.array([int(g) for _, f in terms for (_, g) in f] or [0], dtype=np.int32)
    coef = np.array([[complex(c).real, complex(c).imag] for c, _ in terms] or [[0.0, 0.0]],
                    dtype=np.float64).reshape(-1)
    caps = None if op.get("caps") is None else np.ascontiguousarray(op["caps"], dtype=np.int32)
    keep = (tl, modes, dag, coef, caps)
    d = te_operator_desc()
    d.n_modes, d.n_particles, d.n_terms = L, N, len(terms)
    d.max_occ = caps.ctypes.data_as(C.POINTER(C.c_int32)) if caps is not None else None
    d.term_len = tl.ctypes.data_as(C.POINTER(C.c_int32))
    d.modes = modes.ctypes.data_as(C.POINTER(C.c_int32))
    d.dagger = dag.ctypes.data_as(C.POINTER(C.c_int32))
    d.coef = coef.ctypes.data_as(C.POINTER(C.c_double))
    return d, keep


def te_build_operator(ctx, op: dict):
    desc, keep = operator_desc(op)
    out = C.c_void_p()
    _check(ctx, lib().te_build_operator(ctx, C.byref(desc), C.byref(out)))
    return out


def te_operator_basis_index(op: dict, occ) -> int:
    desc, keep = operator_desc(op)
    o = np.ascontiguousarray(occ, dtype=np.int32)
    idx = C.c_int64()
    s = lib().te_operator_basis_index(C.byref(desc), C.c_void_p(o.ctypes.data), C.byref(idx))
    if s != TE_OK:
        raise TEError(s, "invalid occupation tuple")
    return idx.value


def te_operator_occupation(ctx, op: dict, mode: int, d: int):
    desc, keep = operator_desc(op)
    out = np.empty(d, dtype=np.float64)
    _check(ctx, lib().te_operator_occupation(ctx, C.byref(desc), int(mode),
                                             C.c_void_p(out.ctypes.data), 0))
    return out


def te_model_occupation(ctx, params: dict, mode: int, out=None):
    """Number operator of one mode over the model's basis (numpy array, or fills a
    CUDA float64 tensor given as out)."""
    desc, keep = model_desc(params)
    if out is None:
        info_d = None
        # the dimension follows from the model; build it from the parameters
        if params["model"] in ("tfim", "xxzdm"):
            info_d = 1 << params["L"]
        elif params["model"] == "bose":
            import math
            info_d = math.comb(params["N"] + params["K"] - 1, params["N"])
        else:
            import math
            info_d = (params["N0"] + 1) * math.comb(params["K"] + params["Kp"], params["Nm"])
        out = np.empty(info_d, dtype=np.float64)
    if _is_torch(out):
        ptr, flags = C.c_void_p(out.data_ptr()), TE_PTR_DEVICE if out.is_cuda else 0
    else:
        ptr, flags = C.c_void_p(out.ctypes.data), 0
    _check(ctx, lib().te_model_occupation(ctx, C.byref(desc), int(mode), ptr, flags))
    return out


def te_evolve_sampled(ctx, H, v_in, t: float, t_samples, tol: float, m: int,
                      opt: te_options | None = None, observables=None, want_vectors: bool = True,
                      allow=(TE_OK,)):
    """exp(-iHt) v_in plus the states (and diagonal observables) at t_samples.

    observables: None or an (n_obs, d) float64 array (host) / CUDA tensor.
    Returns (v_out, samples or None, obs_out (n_samples, n_obs) or None,
    sample_bounds, stats dict, status)."""
    d = te_matrix_info_get(H)["d"]
    ip, idev, ik = _vec_ptr(v_in, d)
    ts = np.ascontiguousarray(t_samples, dtype=np.float64)
    ns = ts.size
    if idev:
        import torch
        v_out = torch.empty_like(v_in)
        samples = torch.zeros((ns, d), dtype=torch.complex128, device=v_in.device) if want_vectors else None
    else:
        v_out = np.empty(d, dtype=np.complex128)
        samples = np.zeros((ns, d), dtype=np.complex128) if want_vectors else None
    op = C.c_void_p(v_out.data_ptr() if idev else v_out.ctypes.data)
    sp = C.c_void_p(0)
    if samples is not None:
        sp = C.c_void_p(samples.data_ptr() if idev else samples.ctypes.data)
    nobs = 0
    obp = C.c_void_p(0)
    obs_out = None
    okeep = None
    if observables is not None:
        if idev:
            okeep = observables.contiguous()
            nobs = okeep.shape[0]
            obp = C.c_void_p(okeep.data_ptr())
        else:
            okeep = np.ascontiguousarray(observables, dtype=np.float64)
            nobs = okeep.shape[0]
            obp = C.c_void_p(okeep.ctypes.data)
        obs_out = np.zeros((ns, nobs), dtype=np.float64)
    bounds = np.zeros(ns, dtype=np.float64)
    o = te_options.from_buffer_copy(opt if opt is not None else te_default_options())
    o.flags = (o.flags & ~TE_PTR_DEVICE) | (TE_PTR_DEVICE if idev else 0)
    st = te_stats()
    s = lib().te_evolve_sampled(ctx, H, ip, float(t), ns, C.c_void_p(ts.ctypes.data), float(tol),
                                int(m), C.byref(o), op, sp, nobs, obp,
                                C.c_void_p(obs_out.ctypes.data) if obs_out is not None else C.c_void_p(0),
                                C.c_void_p(bounds.ctypes.data), C.byref(st))
    _check(ctx, s, allow)
    return v_out, samples, obs_out, bounds, st.as_dict(), s


def te_submit(ctx, H, v_in, t: float, tol: float, m: int, opt: te_options | None = None):
    d = te_matrix_info_get(H)["d"]
    ip, idev, ik = _vec_ptr(v_in, d)
    o = te_options.from_buffer_copy(opt if opt is not None else te_default_options())
    o.flags = (o.flags & ~TE_PTR_DEVICE) | (TE_PTR_DEVICE if idev else 0)
    out = C.c_void_p()
    _check(ctx, lib().te_submit(ctx, H, ip, float(t), float(tol), int(m), C.byref(o), C.byref(out)))
    return out


def te_poll(req, v_out=None, d: int | None = None):
    """(status, stats dict); fills v_out (host array or device tensor) when finished."""
    st = te_stats()
    p = C.c_void_p(0)
    keep = None
    if v_out is not None:
        p, _, keep = _vec_ptr(v_out, v_out.shape[0] if d is None else d, writable=True)
    s = lib().te_poll(req, p, C.byref(st))
    return s, st.as_dict()


def te_wait(req, timeout_ms: float = -1.0, v_out=None):
    st = te_stats()
    p = C.c_void_p(0)
    keep = None
    if v_out is not None:
        p, _, keep = _vec_ptr(v_out, v_out.shape[0], writable=True)
    s = lib().te_wait(req, float(timeout_ms), p, C.byref(st))
    return s, st.as_dict()


def te_cancel(req) -> int:
    return lib().te_cancel(req)


def te_request_free(req) -> None:
    lib().te_request_free(req)


def te_set_memory_budget(ctx, nbytes: int) -> None:
    _check(ctx, lib().te_set_memory_budget(ctx, int(nbytes)))


def te_serve_config(ctx, mode: int = 0, m_max: int = 0, capacity: int = 0,
                    large_nnz: int = 0, small_nnz: int = 0) -> None:
    """How te_submit serves requests: TE_SERVE_BATCH (continuous batching) or
    TE_SERVE_SOLO; m_max / capacity shape the serving arenas, large_nnz is the
    large-lane threshold and small_nnz the small batch's (0: keep; negative: none)."""
    _check(ctx, lib().te_serve_config(ctx, int(mode), int(m_max), int(capacity), int(large_nnz),
                                      int(small_nnz)))
