"""ctypes binding of libblcoc.so (include/blcoc.h).  Argument marshalling only: every
step of the solve runs in the library's CUDA kernels.

Low-level functions keep the C names (``blcoc_create``, ``blcoc_solve`` ...) and take
pointers; :class:`Handle` wraps them for torch tensors (device or host) and numpy
arrays (host).  The library must have been built (``paper_1601_05362_gb300.build``);
importing this module without it raises ``RuntimeError`` - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libblcoc.so")

BLCOC_OK = 0
BLCOC_ERR_INVALID_ARG = 1
BLCOC_ERR_NOT_SYMMETRIC = 2
BLCOC_ERR_CUDA = 3
BLCOC_ERR_OOM = 4
BLCOC_NOT_CONVERGED = 5
BLCOC_BREAKDOWN = 6
BLCOC_ERR_TIMEOUT = 7
BLCOC_COCG_RQ = 0
BLCOC_COCR_RQ = 1
BLCOC_COCG_RQ_MIXED = 2
BLCOC_COCR_RQ_MIXED = 3
BLCOC_COCG = 4
BLCOC_COCR = 5
BLCOC_MAX_P = 32
METHODS = {"cocg_rq": BLCOC_COCG_RQ, "cocr_rq": BLCOC_COCR_RQ, "cocg_rq_mixed": BLCOC_COCG_RQ_MIXED,
           "cocr_rq_mixed": BLCOC_COCR_RQ_MIXED, "cocg": BLCOC_COCG, "cocr": BLCOC_COCR}

# name -> (restype, argtypes) for every symbol include/blcoc.h declares
SIGNATURES = {
    "blcoc_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int, C.c_void_p]),
    "blcoc_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int]),
    "blcoc_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.c_void_p, C.c_int]),
    "blcoc_get_xi": (C.c_int, [C.c_void_p, C.c_void_p]),
    "blcoc_spmm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "blcoc_residual_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "blcoc_set_option": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "blcoc_get_stat": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int64)]),
    "blcoc_residual_norm_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "blcoc_set_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "blcoc_sampled_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "blcoc_solve_batched": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                      C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "blcoc_solve_batched_persistent": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                                 C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "blcoc_probe_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "blcoc_destroy": (C.c_int, [C.c_void_p]),
    "blcoc_status_string": (C.c_char_p, [C.c_int]),
    "blcoc_last_error": (C.c_char_p, [C.c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libblcoc.so and bind every declared symbol; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libblcoc.so is not built ({path}); run paper_1601_05362_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BlcocError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s: int) -> str:
    return load_library().blcoc_status_string(int(s)).decode()


# ------------------------------------------------------------------ pointer marshalling
def _ptr(x):
    """(address, keepalive) of a torch tensor or numpy array (contiguous, complex128 or
    the integer CSR types)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if x.is_complex() and (x.is_conj() or x.is_neg()):
                # a lazy conjugate / negative view: its memory does not hold its values
                raise ValueError("tensor is a lazy conj/neg view; pass x.resolve_conj() / x.conj_physical()")
            return x.data_ptr(), x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x)
    return a.ctypes.data, a


def _is_cuda(x) -> bool:
    try:
        import torch
        return isinstance(x, torch.Tensor) and x.is_cuda
    except ImportError:  # pragma: no cover
        return False


def _current_stream(device=None) -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return 0


def _check_block(x, n, name):
    shape = tuple(x.shape)
    if len(shape) != 2 or shape[0] != n:
        raise ValueError(f"{name} must have shape (n, p) with n = {n}, got {shape}")
    dt = str(getattr(x, "dtype", ""))
    if "complex128" not in dt:
        raise ValueError(f"{name} must be complex128, got {dt}")


class Handle:
    """An uploaded matrix A (``blcoc_create``) plus its solve workspace."""

    def __init__(self, n, row_ptr, col_idx, vals, stream=None):
        lib = load_library()
        self._lib = lib
        self.n = int(n)
        self.nnz = int(len(col_idx))
        dev = _is_cuda(row_ptr)
        if dev != _is_cuda(col_idx) or dev != _is_cuda(vals):
            raise ValueError("row_ptr, col_idx and vals must all be host or all be device arrays")
        if not dev:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.complex128)
        p_rp, k1 = _ptr(row_ptr)
        p_ci, k2 = _ptr(col_idx)
        p_va, k3 = _ptr(vals)
        s = _current_stream() if stream is None else int(stream)
        h = C.c_void_p()
        st = lib.blcoc_create(C.byref(h), self.n, self.nnz, p_rp, p_ci, p_va, 0 if dev else 1, s)
        if st != BLCOC_OK:
            raise BlcocError(st, lib.blcoc_last_error(None).decode())
        self._h = h

    @classmethod
    def from_csr(cls, csr, stream=None):
        """From an object with ``n``, ``row_ptr``, ``col_idx``, ``vals`` (host arrays)."""
        return cls(csr.n, csr.row_ptr, csr.col_idx, csr.vals, stream=stream)

    # -------------------------------------------------------------- solve
    def solve(self, B, X, method="cocr_rq", tol=1e-10, maxit=None, check=True):
        """Run bl_cocg_rq / bl_cocr_rq; X (n x p) is the initial guess and receives the
        result.  Returns the status code (raises on errors when ``check``; convergence
        failure and breakdown are returned, not raised)."""
        _check_block(B, self.n, "B")
        _check_block(X, self.n, "X")
        p = int(B.shape[1])
        if tuple(X.shape) != tuple(B.shape):
            raise ValueError("X and B must have the same shape")
        maxit = self.n if maxit is None else int(maxit)
        pb, kb = _ptr(B)
        px, kx = _ptr(X)
        if not _is_cuda(X) and isinstance(X, np.ndarray) and kx is not X:
            raise ValueError("host X must be a contiguous numpy array (it is written in place)")
        st = self._lib.blcoc_solve(self._h, pb, px, p, METHODS[method] if isinstance(method, str) else int(method),
                                   float(tol), maxit)
        if check and st not in (BLCOC_OK, BLCOC_NOT_CONVERGED, BLCOC_BREAKDOWN):
            raise BlcocError(st, self.last_error())
        return st

    def info(self, hist_len=None):
        it = C.c_int()
        rr = C.c_double()
        rt = C.c_double()
        self._lib.blcoc_get_info(self._h, C.byref(it), C.byref(rr), C.byref(rt), None, 0)
        k = it.value + 1 if hist_len is None else int(hist_len)
        hist = np.zeros(max(k, 1), dtype=np.float64)
        self._lib.blcoc_get_info(self._h, None, None, None, hist.ctypes.data, hist.shape[0])
        return {"iters": it.value, "relres": rr.value, "relres_true": rt.value, "hist": hist[:k]}

    def xi(self, p):
        out = np.zeros((p, p), dtype=np.complex128)
        st = self._lib.blcoc_get_xi(self._h, out.ctypes.data)
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())
        return out

    def spmm(self, X, Y):
        _check_block(X, self.n, "X")
        _check_block(Y, self.n, "Y")
        px, kx = _ptr(X)
        py, ky = _ptr(Y)
        st = self._lib.blcoc_spmm(self._h, px, py, int(X.shape[1]))
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())

    def residual_norm(self, B, X):
        _check_block(B, self.n, "B")
        _check_block(X, self.n, "X")
        pb, kb = _ptr(B)
        px, kx = _ptr(X)
        out = C.c_double()
        st = self._lib.blcoc_residual_norm(self._h, pb, px, int(B.shape[1]), C.byref(out))
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())
        return out.value

    def set_values(self, vals):
        """Replace A's values (same pattern); torch device tensor or host array."""
        if len(vals) != self.nnz:
            raise ValueError("vals must have nnz entries")
        dev = _is_cuda(vals)
        if not dev:
            vals = np.ascontiguousarray(vals, dtype=np.complex128)
        pv, kv = _ptr(vals)
        st = self._lib.blcoc_set_values(self._h, pv, 0 if dev else 1)
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())

    def sampled_grad(self, Lam, X, out):
        """out[e] = -sum_k Lam[i,k] conj(X[j,k]) over the stored entries (device tensors)."""
        _check_block(Lam, self.n, "Lambda")
        _check_block(X, self.n, "X")
        pl, kl = _ptr(Lam)
        px, kx = _ptr(X)
        po, ko = _ptr(out)
        st = self._lib.blcoc_sampled_grad(self._h, pl, px, int(X.shape[1]), po)
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())

    def set_option(self, key: str, value: int):
        st = self._lib.blcoc_set_option(self._h, key.encode(), int(value))
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())

    def stat(self, key: str) -> int:
        v = C.c_int64()
        st = self._lib.blcoc_get_stat(self._h, key.encode(), C.byref(v))
        if st != BLCOC_OK:
            raise BlcocError(st, self.last_error())
        return v.value

    def last_error(self) -> str:
        return self._lib.blcoc_last_error(self._h).decode()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.blcoc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batched(handles, Bs, Xs, method="cocr_rq", tol=1e-10, maxit=None, autotune=True, persistent=False):
    """blcoc_solve_batched (or, with persistent=True, blcoc_solve_batched_persistent) over
    lists of Handles and device tensors; returns (status, ms per system-iteration, launch
    shape message)."""
    lib = load_library()
    k = len(handles)
    if not (len(Bs) == len(Xs) == k):
        raise ValueError("handles, Bs and Xs must have the same length")
    for h, b, x in zip(handles, Bs, Xs):
        _check_block(b, h.n, "B")
        _check_block(x, h.n, "X")
        if not (_is_cuda(b) and _is_cuda(x)):
            raise ValueError("batched solves take device tensors")
    hs = (C.c_void_p * k)(*[h._h.value for h in handles])
    bp = (C.c_void_p * k)(*[_ptr(b)[0] for b in Bs])
    xp = (C.c_void_p * k)(*[_ptr(x)[0] for x in Xs])
    ps = (C.c_int * k)(*[int(b.shape[1]) for b in Bs])
    maxit = max(h.n for h in handles) if maxit is None else int(maxit)
    ms = C.c_double()
    fn = lib.blcoc_solve_batched_persistent if persistent else lib.blcoc_solve_batched
    st = fn(k, hs, bp, xp, ps, METHODS[method] if isinstance(method, str) else int(method),
            float(tol), maxit, 1 if autotune else 0, C.byref(ms))
    msg = lib.blcoc_last_error(hs[0]).decode() if k else ""
    if st not in (BLCOC_OK, BLCOC_NOT_CONVERGED, BLCOC_BREAKDOWN):
        raise BlcocError(st, msg or lib.blcoc_last_error(None).decode())
    return st, ms.value, msg


def probe_peak(kind: str = "fp64") -> float:
    """blcoc_probe_peak: measured FMA throughput of the current device in flop/s
    (kind "fp64" or "fp32")."""
    lib = load_library()
    v = C.c_double()
    st = lib.blcoc_probe_peak({"fp64": 0, "fp32": 1}[kind], C.byref(v))
    if st != BLCOC_OK:
        raise BlcocError(st, lib.blcoc_last_error(None).decode())
    return v.value


# ------------------------------------------------------------------ same names as the ABI
def blcoc_create(n, row_ptr, col_idx, vals, stream=None) -> Handle:
    return Handle(n, row_ptr, col_idx, vals, stream=stream)


def blcoc_solve(h: Handle, B, X, method="cocr_rq", tol=1e-10, maxit=None) -> int:
    return h.solve(B, X, method=method, tol=tol, maxit=maxit)


def blcoc_get_info(h: Handle):
    return h.info()


def blcoc_destroy(h: Handle) -> None:
    h.close()
