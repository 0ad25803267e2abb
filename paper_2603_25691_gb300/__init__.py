"""GB300 (sm_103a) solver for the unaligned kernel-mode CP-HIFI subproblem.

Python binding of ``libcphifi.so``: argument marshalling only.  Every step of
the solve runs in the library's CUDA kernels; there is no CPU fallback and
importing the functions below raises when the shared library is missing.

Host buffers are NumPy arrays; device buffers are CUDA ``torch.Tensor`` s.
n x r matrices are column-major (the paper's vec order) on both sides: pass
NumPy arrays of shape (n, r) (they are converted to Fortran order) or
device tensors holding the column-major data (``to_colmajor`` builds one).
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcphifi.so")

OK = 0
E_INVALID_ARG = 1
E_OOM = 2
E_ADMISSION = 3
E_NOT_CONVERGED = 4
E_BREAKDOWN = 5
E_DEVICE = 6
E_TIMEOUT = 7
E_UNSUPPORTED = 8

MEM_HOST = 0
MEM_DEVICE = 1

FP64 = 0
MIXED_FP32 = 1
MIXED_TF32 = 2
MIXED_BF16 = 3
FP64_EMULATED = 4
MIXED_TF32X3 = 5
MIXED_BF16X3 = 6

OBS_SORTED = 0x1
NEED_LOWP = 0x4

PRECISIONS = {"fp64": FP64, "mixed_fp32": MIXED_FP32, "mixed_tf32": MIXED_TF32,
              "mixed_bf16": MIXED_BF16, "fp64_emulated": FP64_EMULATED,
              "mixed_tf32x3": MIXED_TF32X3, "mixed_bf16x3": MIXED_BF16X3}
NEED_FP64 = 0x2
KEEP_OBS = 0x8
VALS_F32 = 0x10


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("rho", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("k_replace", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("gram", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("true_residuals", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("rel_residual_recurrence", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("gds_ms", ctypes.c_double), ("gds_launches", ctypes.c_int32),
                ("gemm_launches", ctypes.c_int32), ("gemm_ms", ctypes.c_double),
                ("gds64_ms", ctypes.c_double), ("gds64_launches", ctypes.c_int32),
                ("gemm64_launches", ctypes.c_int32), ("gemm64_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("setup_launches", ctypes.c_int64),
                ("rhs_ms", ctypes.c_double), ("iter_ms", ctypes.c_double),
                ("final_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("graph_build_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("gds_warps_per_sm", ctypes.c_int32), ("split32", ctypes.c_int32),
                ("split_tc", ctypes.c_int32), ("split_wide", ctypes.c_int32),
                ("split64", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class BatchItem(ctypes.Structure):
    _fields_ = [("kern", ctypes.c_void_p), ("d_other", ctypes.c_int32), ("r", ctypes.c_int32),
                ("other_sizes", ctypes.c_void_p), ("factors", ctypes.c_void_p),
                ("q", ctypes.c_int64), ("kidx", ctypes.c_void_p), ("oidx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("hold", ctypes.c_uint32), ("W_out", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("create_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("tiles", ctypes.c_int64),
                ("blocks", ctypes.c_int32), ("timed_out", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class CphifiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cphifi status {status}: {msg}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_SIG = {
    "cphifi_ctx_create": (ctypes.c_int, [_PP, ctypes.c_int, ctypes.c_size_t]),
    "cphifi_ctx_destroy": (ctypes.c_int, [_P]),
    "cphifi_ctx_set_stream": (ctypes.c_int, [_P, _P]),
    "cphifi_ctx_bytes_in_use": (ctypes.c_size_t, [_P]),
    "cphifi_last_error": (ctypes.c_char_p, [_P]),
    "cphifi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cphifi_kernel_create": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_int, _PP]),
    "cphifi_kernel_destroy": (ctypes.c_int, [_P]),
    "cphifi_kernel_eig": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "cphifi_kernel_create_points": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P,
                                                   ctypes.c_int32, ctypes.c_double, ctypes.c_int,
                                                   _PP]),
    "cphifi_kernel_apply": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                           ctypes.c_int]),
    "cphifi_problem_create": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                             ctypes.c_int64, _P, _P, _P, ctypes.c_uint32,
                                             ctypes.c_int, _PP]),
    "cphifi_problem_destroy": (ctypes.c_int, [_P]),
    "cphifi_problem_bytes": (ctypes.c_size_t, [_P]),
    "cphifi_problem_solve": (ctypes.c_int, [_P, ctypes.POINTER(Params), _P, _P, ctypes.c_int,
                                            ctypes.POINTER(Stats)]),
    "cphifi_solve": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                    ctypes.c_int64, _P, _P, _P, ctypes.c_uint32,
                                    ctypes.POINTER(Params), _P, _P, ctypes.c_int,
                                    ctypes.POINTER(Stats)]),
    "cphifi_problem_rhs": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "cphifi_problem_matvec": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             _P, _P, ctypes.c_int]),
    "cphifi_problem_gds": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "cphifi_problem_precond": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, _P,
                                              ctypes.c_int]),
    "cphifi_problem_gram": (ctypes.c_int, [_P, _P, _P, _P]),
    "cphifi_problem_grams": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "cphifi_problem_order": (ctypes.c_int, [_P, _P, _P]),
    "cphifi_ctx_set_slots": (ctypes.c_int, [_P, ctypes.c_int]),
    "cphifi_ctx_set_batch_wait": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cphifi_ctx_set_tuning": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(Tuning)]),
    "cphifi_problem_set_factors": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "cphifi_problem_update_factor": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int]),
    "cphifi_problem_fit": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "cphifi_als": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int64,
                                  _P, _P, _P, ctypes.c_uint32, ctypes.POINTER(Params),
                                  ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                  ctypes.POINTER(Stats)]),
    "cphifi_submit": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                     ctypes.c_int64, _P, _P, _P, ctypes.c_uint32,
                                     ctypes.POINTER(Params), _P, _P, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "cphifi_poll": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32)]),
    "cphifi_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(Stats)]),
    "cphifi_solve_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BatchItem),
                                          ctypes.POINTER(Params), ctypes.c_int,
                                          ctypes.POINTER(Stats), ctypes.POINTER(BatchInfo)]),
    "cphifi_gds_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                          ctypes.c_int64, _P, _P, _P,
                                          ctypes.POINTER(ctypes.c_char_p)]),
}


def exported_symbols() -> list:
    """Names of the C entry points this binding expects (all of include/cphifi.h)."""
    return list(_SIG)


def lib():
    """Load libcphifi.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().cphifi_status_string(code).decode()


# --------------------------------------------------------------- buffers ---
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class _Buf:
    """Keeps a host array or device tensor alive and yields (pointer, kind)."""

    def __init__(self, x, dtype, shape_check=None, colmajor=False):
        if _is_torch(x):
            import torch
            want = {np.float64: torch.float64, np.float32: torch.float32,
                    np.int32: torch.int32}[dtype]
            if not x.is_cuda:
                x = x.numpy()
            else:
                if x.dtype != want:
                    raise TypeError(f"device buffer must be {want}, got {x.dtype}")
                if not x.is_contiguous():
                    raise ValueError("device buffers must be contiguous")
                self.obj, self.ptr, self.mem = x, x.data_ptr(), MEM_DEVICE
                self.numel = x.numel()
                return
        a = np.asarray(x, dtype=dtype)
        a = np.asfortranarray(a) if colmajor else np.ascontiguousarray(a)
        self.obj, self.ptr, self.mem = a, a.ctypes.data, MEM_HOST
        self.numel = a.size


def to_colmajor(X):
    """(n, r) torch tensor -> contiguous tensor holding its column-major data."""
    return X.t().contiguous()


def _check(ctx_ptr, rc: int, what: str):
    if rc != OK:
        msg = lib().cphifi_last_error(ctx_ptr).decode() if ctx_ptr else status_string(rc)
        raise CphifiError(rc, f"{what}: {msg}")


# ---------------------------------------------------------------- handles ---
class Context:
    """cphifi_ctx_create / cphifi_ctx_destroy."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        rc = lib().cphifi_ctx_create(ctypes.byref(h), device, hbm_budget_bytes)
        _check(None, rc, "ctx_create")
        self.h = h
        # kernels and problems created on this context, destroyed before it
        self._children = weakref.WeakSet()

    def set_stream(self, stream) -> None:
        """cphifi_ctx_set_stream: order calls on a torch.cuda.Stream or raw handle."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(self.h, lib().cphifi_ctx_set_stream(self.h, ctypes.c_void_p(handle)),
               "ctx_set_stream")

    def bytes_in_use(self) -> int:
        return lib().cphifi_ctx_bytes_in_use(self.h)

    def last_error(self) -> str:
        return lib().cphifi_last_error(self.h).decode()

    def close(self):
        """Destroys the problems and kernels still open on this context, then
        the context (their handles are dead afterwards)."""
        if getattr(self, "h", None):
            children = list(getattr(self, "_children", ()))
            for ch in sorted(children, key=lambda c: isinstance(c, Kernel)):
                try:
                    ch.close()
                except CphifiError:
                    ch.h = None
            lib().cphifi_ctx_destroy(self.h)
            self.h = None

    __del__ = close

    def set_tuning(self, bucket, shapes) -> None:
        """cphifi_ctx_set_tuning: launch shapes (a dict with the fields of
        Tuning, missing ones 0 = heuristic; None removes the entry) for the
        size bucket (floor(log2 n), floor(log2 q), r), see size_bucket()."""
        n_log2, q_log2, r = (int(x) for x in bucket)
        if shapes is None:
            rc = lib().cphifi_ctx_set_tuning(self.h, n_log2, q_log2, r, None)
        else:
            t = Tuning(*[int(shapes.get(f, 0)) for f, _ in Tuning._fields_[:5]])
            rc = lib().cphifi_ctx_set_tuning(self.h, n_log2, q_log2, r, ctypes.byref(t))
        _check(self.h, rc, "ctx_set_tuning")

    def set_slots(self, max_active: int) -> None:
        """cphifi_ctx_set_slots: how many submitted requests run at once."""
        _check(self.h, lib().cphifi_ctx_set_slots(self.h, int(max_active)), "ctx_set_slots")

    def set_batch_wait(self, ms: int) -> None:
        """cphifi_ctx_set_batch_wait: the persistent launch's idle-wait bound."""
        _check(self.h, lib().cphifi_ctx_set_batch_wait(self.h, int(ms)), "ctx_set_batch_wait")

    def poll(self, done_cap: int = 0):
        """cphifi_poll: advance all submitted requests.  Returns (active,
        pending), or (active, pending, completed tickets) when done_cap > 0."""
        a, p, nd = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        buf = (ctypes.c_uint64 * max(done_cap, 1))()
        _check(self.h, lib().cphifi_poll(self.h, ctypes.byref(a), ctypes.byref(p), buf,
                                         int(done_cap), ctypes.byref(nd)), "poll")
        if done_cap > 0:
            return a.value, p.value, list(buf[:nd.value])
        return a.value, p.value

    def kernel_create(self, n: int, UK, DK, K=None) -> "Kernel":
        return Kernel(self, n, UK, DK, K)

    def kernel_from_points(self, x, kind: str = "gaussian", bandwidth: float = 0.1) -> "Kernel":
        """cphifi_kernel_create_points: K(i, j) = k(x_i, x_j) for the points x
        (n values, or an n x dim array), kind "gaussian" or "matern32"."""
        return Kernel.from_points(self, x, kind, bandwidth)


class Kernel:
    """cphifi_kernel_create: the kernel matrix's eigendecomposition (Eq. eigK)."""

    def __init__(self, ctx: Context, n: int, UK, DK, K=None):
        # UK = DK = None: the library computes eig(K) on the device from K.
        self.ctx = ctx
        self.n = int(n)
        h = ctypes.c_void_p()
        if UK is None and DK is None:
            if K is None:
                raise ValueError("pass K or its eigendecomposition (UK, DK)")
            k = _Buf(K, np.float64, colmajor=True)
            if k.numel != self.n * self.n:
                raise ValueError("K must be n x n")
            rc = lib().cphifi_kernel_create(ctx.h, self.n, k.ptr, None, None, k.mem,
                                            ctypes.byref(h))
            _check(ctx.h, rc, "kernel_create")
            self.h = h
            ctx._children.add(self)
            return
        u = _Buf(UK, np.float64, colmajor=True)
        d = _Buf(DK, np.float64)
        if u.mem != d.mem:
            raise ValueError("UK and DK must live in the same memory kind")
        if u.numel != self.n * self.n or d.numel != self.n:
            raise ValueError("UK must be n x n and DK length n")
        rc = lib().cphifi_kernel_create(ctx.h, self.n, None, u.ptr, d.ptr, u.mem, ctypes.byref(h))
        _check(ctx.h, rc, "kernel_create")
        self.h = h
        ctx._children.add(self)

    @classmethod
    def from_points(cls, ctx: Context, x, kind: str = "gaussian", bandwidth: float = 0.1):
        pts = np.asarray(x, dtype=np.float64)
        if pts.ndim == 1:
            pts = pts[:, None]
        pts = np.ascontiguousarray(pts)
        self = cls.__new__(cls)
        self.ctx, self.n = ctx, int(pts.shape[0])
        h = ctypes.c_void_p()
        kinds = {"gaussian": 0, "matern32": 1}
        rc = lib().cphifi_kernel_create_points(ctx.h, self.n, int(pts.shape[1]), pts.ctypes.data,
                                               kinds[kind], float(bandwidth), MEM_HOST,
                                               ctypes.byref(h))
        _check(ctx.h, rc, "kernel_create_points")
        self.h = h
        ctx._children.add(self)
        return self

    def apply(self, X, precision: str = "fp64"):
        """cphifi_kernel_apply: K X for an (n, r) host array."""
        X = np.asfortranarray(np.asarray(X, dtype=np.float64))
        Y = np.empty_like(X, order="F")
        _check(self.ctx.h, lib().cphifi_kernel_apply(self.h, _prec(precision), int(X.shape[1]),
                                                     X.ctypes.data, Y.ctypes.data, MEM_HOST),
               "kernel_apply")
        return Y

    def eig(self):
        """cphifi_kernel_eig: (D_K, U_K) held by the handle, as host arrays."""
        U = np.empty((self.n, self.n), order="F")
        d = np.empty(self.n)
        _check(self.ctx.h, lib().cphifi_kernel_eig(self.h, U.ctypes.data, d.ctypes.data,
                                                   MEM_HOST), "kernel_eig")
        return d, U

    def close(self):
        """cphifi_kernel_destroy (raises while submitted requests still use it)."""
        if getattr(self, "h", None) and not getattr(self.ctx, "h", None):
            self.h = None  # the context is gone, and the kernel with it
        if getattr(self, "h", None):
            rc = lib().cphifi_kernel_destroy(self.h)
            _check(self.ctx.h, rc, "kernel_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _factor_bufs(factors, r):
    bufs = [_Buf(F, np.float64, colmajor=True) for F in factors]
    sizes = []
    for F, b in zip(factors, bufs):
        sizes.append(int(F.shape[0]) if b.mem == MEM_HOST else b.numel // r)
    return bufs, sizes


def _vals_f32(vals) -> bool:
    """FP32 observation values (numpy or torch float32) go to the library as
    they are, with the CPHIFI_VALS_F32 flag; anything else as FP64."""
    return str(getattr(vals, "dtype", "")) in ("float32", "torch.float32")


def _obs_bufs(kidx, oidx, vals):
    k = _Buf(kidx, np.int32)
    o = _Buf(oidx, np.int32)
    v = _Buf(vals, np.float32 if _vals_f32(vals) else np.float64)
    if not (k.mem == o.mem == v.mem):
        raise ValueError("observation lists must live in the same memory kind")
    return k, o, v


def _vals_flag(vals) -> int:
    return VALS_F32 if _vals_f32(vals) else 0


class Problem:
    """cphifi_problem_create: one subproblem (sort, Zhat, Gram, eig(V), B)."""

    def __init__(self, ctx: Context, kernel: Kernel, factors, kidx, oidx, vals, r: int,
                 sorted_obs: bool = False, lowp: bool | None = None, keep_obs: bool = False):
        # lowp: True = build only the hi/lo data of the mixed/emulated modes,
        # False = only the FP64 data, None = both.  keep_obs: keep the sorted
        # observation lists (needed by the alternating-fit calls).
        self.ctx, self.kernel, self.r = ctx, kernel, int(r)
        self.n = kernel.n
        fb, sizes = _factor_bufs(factors, self.r)
        k, o, v = _obs_bufs(kidx, oidx, vals)
        if any(b.mem != k.mem for b in fb):
            raise ValueError("factors and observations must live in the same memory kind")
        self.q = k.numel
        self.d_other = len(factors)
        self.sizes = sizes
        sizes_arr = (ctypes.c_int64 * len(sizes))(*sizes)
        fptrs = (ctypes.c_void_p * len(fb))(*[b.ptr for b in fb])
        flags = (OBS_SORTED if sorted_obs else 0) | (KEEP_OBS if keep_obs else 0) | \
            _vals_flag(vals)
        if lowp is True:
            flags |= NEED_LOWP
        elif lowp is False:
            flags |= NEED_FP64
        h = ctypes.c_void_p()
        rc = lib().cphifi_problem_create(ctx.h, kernel.h, len(fb), sizes_arr, fptrs, self.r,
                                         self.q, k.ptr, o.ptr, v.ptr, flags, k.mem,
                                         ctypes.byref(h))
        _check(ctx.h, rc, "problem_create")
        self.h = h
        ctx._children.add(self)
        self.mem = k.mem

    def close(self):
        if getattr(self, "h", None) and getattr(getattr(self, "ctx", None), "h", None):
            lib().cphifi_problem_destroy(self.h)
        self.h = None

    __del__ = close

    def bytes(self) -> int:
        return lib().cphifi_problem_bytes(self.h)

    # ---- outputs: host numpy (n, r) or a device tensor (flat, column-major)
    def _out(self, like_device: bool):
        if like_device:
            import torch
            return torch.empty(self.n * self.r, dtype=torch.float64, device="cuda")
        return np.empty((self.n, self.r), dtype=np.float64, order="F")

    def solve(self, lam: float, rho: float, tol: float, max_iter: int = 1000,
              precision: str | int = "fp64", k_replace: int = 10, check_every: int = 8,
              profile: bool = False, W0=None, out=None, raise_on_error: bool = True,
              gram: int = 0):
        """cphifi_problem_solve.  Returns (W, stats dict)."""
        prm = make_params(lam, rho, tol, max_iter, precision, k_replace, check_every, profile,
                          gram)
        st = Stats()
        W = out if out is not None else self._out(False)
        wb = _Buf(W, np.float64, colmajor=True) if not _is_torch(W) else _Buf(W, np.float64)
        w0 = _Buf(W0, np.float64, colmajor=True) if W0 is not None else None
        rc = lib().cphifi_problem_solve(self.h, ctypes.byref(prm), w0.ptr if w0 else None,
                                        wb.ptr, wb.mem, ctypes.byref(st))
        if rc not in (OK, E_NOT_CONVERGED) or (raise_on_error and rc != OK):
            _check(self.ctx.h, rc, "problem_solve")
        return (wb.obj if wb.mem == MEM_DEVICE else wb.obj), st.as_dict()

    def rhs(self):
        """cphifi_problem_rhs: (B, b) as (n, r) host arrays."""
        B = self._out(False)
        b = self._out(False)
        _check(self.ctx.h, lib().cphifi_problem_rhs(self.h, B.ctypes.data, b.ctypes.data, MEM_HOST),
               "problem_rhs")
        return B, b

    def matvec(self, X, lam: float, rho: float, precision: str | int = "fp64"):
        """cphifi_problem_matvec: Y = A X in the given operator arithmetic."""
        x = _Buf(X, np.float64, colmajor=True)
        Y = self._out(False)
        _check(self.ctx.h, lib().cphifi_problem_matvec(self.h, _prec(precision), lam, rho, x.ptr,
                                                       Y.ctypes.data, MEM_HOST), "problem_matvec")
        return Y

    def gds(self, Xhat, precision: str | int = "fp64"):
        """cphifi_problem_gds: Yhat1 for a given Xhat (Eqs. vl and yhat1)."""
        x = _Buf(Xhat, np.float64, colmajor=True)
        Y = self._out(False)
        _check(self.ctx.h, lib().cphifi_problem_gds(self.h, _prec(precision), x.ptr, Y.ctypes.data,
                                                    MEM_HOST), "problem_gds")
        return Y

    def precond(self, X, lam: float, rho: float):
        """cphifi_problem_precond: M^{-1} X (Eq. fx)."""
        x = _Buf(X, np.float64, colmajor=True)
        Y = self._out(False)
        _check(self.ctx.h, lib().cphifi_problem_precond(self.h, lam, rho, x.ptr, Y.ctypes.data,
                                                        MEM_HOST), "problem_precond")
        return Y

    def grams(self, precision: str | int = "fp64"):
        """cphifi_problem_grams: the per-index Gram blocks, an (n, r, r) array."""
        C = np.empty((self.n, self.r, self.r))
        _check(self.ctx.h, lib().cphifi_problem_grams(self.h, _prec(precision), C.ctypes.data,
                                                      MEM_HOST), "problem_grams")
        return C

    def gram(self):
        """cphifi_problem_gram: (V, DV, UV) computed on the device."""
        r = self.r
        V = np.empty((r, r), order="F")
        DV = np.empty(r)
        UV = np.empty((r, r), order="F")
        _check(self.ctx.h, lib().cphifi_problem_gram(self.h, V.ctypes.data, DV.ctypes.data,
                                                     UV.ctypes.data), "problem_gram")
        return V, DV, UV

    def set_factors(self, factors) -> None:
        """cphifi_problem_set_factors: new finite factors (host arrays)."""
        fb = [_Buf(F, np.float64, colmajor=True) for F in factors]
        fptrs = (ctypes.c_void_p * len(fb))(*[b.ptr for b in fb])
        _check(self.ctx.h, lib().cphifi_problem_set_factors(self.h, fptrs, MEM_HOST),
               "problem_set_factors")

    def update_factor(self, mode: int, W):
        """cphifi_problem_update_factor: the CP-ALS update of finite mode
        `mode` for weights W; returns the new factor (n_m, r)."""
        w = _Buf(W, np.float64, colmajor=True)
        A = np.empty((self.sizes[mode], self.r), order="F")
        _check(self.ctx.h, lib().cphifi_problem_update_factor(self.h, int(mode), w.ptr,
                                                              A.ctypes.data, MEM_HOST),
               "problem_update_factor")
        return A

    def fit(self, W):
        """cphifi_problem_fit: (sum (t - m)^2, sum t^2) of the model K W."""
        w = _Buf(W, np.float64, colmajor=True)
        r2, t2 = ctypes.c_double(), ctypes.c_double()
        _check(self.ctx.h, lib().cphifi_problem_fit(self.h, w.ptr, MEM_HOST, ctypes.byref(r2),
                                                    ctypes.byref(t2)), "problem_fit")
        return r2.value, t2.value

    def order(self):
        """cphifi_problem_order: (perm, row_ptr) of the stable sort by kernel index."""
        perm = np.empty(self.q, dtype=np.int32)
        rp = np.empty(self.n + 1, dtype=np.int64)
        _check(self.ctx.h, lib().cphifi_problem_order(self.h, perm.ctypes.data, rp.ctypes.data),
               "problem_order")
        return perm, rp


GRAM_FORM = 0x100


def size_bucket(n: int, q: int, r: int):
    """The tuning bucket of a problem: (floor(log2 n), floor(log2 max(q, 1)), r)."""
    return (int(n).bit_length() - 1, max(int(q), 1).bit_length() - 1, int(r))


def _prec(p) -> int:
    """Precision name or code; a '+gram' suffix adds CPHIFI_GRAM_FORM (step
    calls: the product from the per-index Gram blocks)."""
    if isinstance(p, str):
        base, _, form = p.partition("+")
        return PRECISIONS[base] | (GRAM_FORM if form == "gram" else 0)
    return int(p)


def make_params(lam, rho, tol, max_iter=1000, precision="fp64", k_replace=10, check_every=8,
                profile=False, gram=0) -> Params:
    return Params(float(lam), float(rho), float(tol), int(max_iter), _prec(precision),
                  int(k_replace), int(check_every), 1 if profile else 0, int(gram))


def solve(ctx: Context, kernel: Kernel, factors, kidx, oidx, vals, r: int, lam: float, rho: float,
          tol: float, max_iter: int = 1000, precision="fp64", sorted_obs=False, k_replace=10,
          check_every=8, profile=False, W0=None, out=None, gram=0):
    """cphifi_solve: one-shot create + solve + destroy.  Returns (W, stats)."""
    fb, sizes = _factor_bufs(factors, r)
    k, o, v = _obs_bufs(kidx, oidx, vals)
    prm = make_params(lam, rho, tol, max_iter, precision, k_replace, check_every, profile, gram)
    st = Stats()
    n = kernel.n
    if out is None:
        out = np.empty((n, r), order="F") if k.mem == MEM_HOST else None
        if out is None:
            import torch
            out = torch.empty(n * r, dtype=torch.float64, device="cuda")
    wb = _Buf(out, np.float64, colmajor=not _is_torch(out))
    w0 = _Buf(W0, np.float64, colmajor=True) if W0 is not None else None
    sizes_arr = (ctypes.c_int64 * len(sizes))(*sizes)
    fptrs = (ctypes.c_void_p * len(fb))(*[b.ptr for b in fb])
    flags = (OBS_SORTED if sorted_obs else 0) | _vals_flag(vals)
    rc = lib().cphifi_solve(ctx.h, kernel.h, len(fb), sizes_arr, fptrs, int(r), k.numel, k.ptr,
                            o.ptr, v.ptr, flags, ctypes.byref(prm), w0.ptr if w0 else None,
                            wb.ptr, k.mem, ctypes.byref(st))
    if rc not in (OK, E_NOT_CONVERGED):
        _check(ctx.h, rc, "solve")
    return wb.obj, st.as_dict()


def als(ctx: Context, kernel: Kernel, factors, kidx, oidx, vals, r: int, lam: float, rho: float,
        tol: float, sweeps: int, als_tol: float = 0.0, max_iter: int = 1000, precision="fp64",
        sorted_obs=False, k_replace=10, check_every=8, W0=None):
    """cphifi_als on host arrays: the alternating fit (§2).  `factors` is the
    start; returns (W, fitted factors, fit errors per sweep, last solve's stats)."""
    facs = [np.array(F, dtype=np.float64, order="F") for F in factors]
    k, o, v = _obs_bufs(kidx, oidx, vals)
    if k.mem != MEM_HOST:
        raise ValueError("als() takes host arrays")
    n = kernel.n
    W = np.zeros((n, r), order="F") if W0 is None else np.array(W0, dtype=np.float64, order="F")
    sizes = [F.shape[0] for F in facs]
    sizes_arr = (ctypes.c_int64 * len(sizes))(*sizes)
    fptrs = (ctypes.c_void_p * len(facs))(*[F.ctypes.data for F in facs])
    prm = make_params(lam, rho, tol, max_iter, precision, k_replace, check_every, False)
    errs = np.zeros(sweeps)
    done = ctypes.c_int32()
    st = Stats()
    rc = lib().cphifi_als(ctx.h, kernel.h, len(facs), sizes_arr, fptrs, int(r), k.numel, k.ptr,
                          o.ptr, v.ptr, (OBS_SORTED if sorted_obs else 0) | _vals_flag(vals),
                          ctypes.byref(prm),
                          int(sweeps), float(als_tol), 1 if W0 is not None else 0,
                          W.ctypes.data, errs.ctypes.data, ctypes.byref(done), MEM_HOST,
                          ctypes.byref(st))
    _check(ctx.h, rc, "als")
    return W, facs, errs[:done.value], st.as_dict()


class Request:
    """A submitted solve (cphifi_submit); keeps its buffers alive until wait()."""

    def __init__(self, ctx, ticket, bufs, out):
        self.ctx, self.ticket, self._bufs, self.out = ctx, ticket, bufs, out
        self.result = None

    def wait(self, timeout_us: int = -1):
        """cphifi_wait: returns (W, stats); raises CphifiError(E_TIMEOUT) if
        the request is still running after `timeout_us` (it keeps running)."""
        if self.result is not None:
            return self.result
        st = Stats()
        rc = lib().cphifi_wait(self.ctx.h, ctypes.c_uint64(self.ticket), int(timeout_us),
                               ctypes.byref(st))
        if rc == E_TIMEOUT:
            _check(self.ctx.h, rc, "wait")
        self._bufs = None
        self.result = (self.out, st.as_dict())
        if rc not in (OK, E_NOT_CONVERGED):
            _check(self.ctx.h, rc, "request")
        return self.result


def submit(ctx: Context, kernel: Kernel, factors, kidx, oidx, vals, r: int, lam: float,
           rho: float, tol: float, max_iter: int = 1000, precision="fp64", sorted_obs=False,
           k_replace=10, check_every=8, W0=None, out=None, gram=0) -> Request:
    """cphifi_submit: queue one solve; returns a Request whose wait() gives (W, stats)."""
    fb, sizes = _factor_bufs(factors, r)
    k, o, v = _obs_bufs(kidx, oidx, vals)
    prm = make_params(lam, rho, tol, max_iter, precision, k_replace, check_every, False, gram)
    n = kernel.n
    if out is None:
        out = np.empty((n, r), order="F") if k.mem == MEM_HOST else None
        if out is None:
            import torch
            out = torch.empty(n * r, dtype=torch.float64, device="cuda")
    wb = _Buf(out, np.float64, colmajor=not _is_torch(out))
    w0 = _Buf(W0, np.float64, colmajor=True) if W0 is not None else None
    sizes_arr = (ctypes.c_int64 * len(sizes))(*sizes)
    fptrs = (ctypes.c_void_p * len(fb))(*[b.ptr for b in fb])
    flags = (OBS_SORTED if sorted_obs else 0) | _vals_flag(vals)
    t = ctypes.c_uint64()
    rc = lib().cphifi_submit(ctx.h, kernel.h, len(fb), sizes_arr, fptrs, int(r), k.numel, k.ptr,
                             o.ptr, v.ptr, flags, ctypes.byref(prm), w0.ptr if w0 else None,
                             wb.ptr, k.mem, ctypes.byref(t))
    _check(ctx.h, rc, "submit")
    # the request keeps its buffers and the kernel handle alive until wait()
    return Request(ctx, t.value, (kernel, fb, k, o, v, wb, w0, sizes_arr, fptrs, prm), wb.obj)


def solve_batch(ctx: Context, problems, lam: float, rho: float, tol: float, max_iter: int = 1000,
                k_replace=10, precision="mixed_fp32"):
    """cphifi_solve_batch: many mixed-FP32 solves in one persistent launch.

    problems: a list of dicts with keys kernel, factors, kidx, oidx, vals, r
    and optionally sorted_obs, out (W's storage) and hold (True: the item is
    never started, so the launch ends by its bounded wait); all host arrays,
    or all device tensors.
    Returns (list of W, list of stats dicts, launch info dict); a solve that
    did not converge has its status in its stats."""
    prm = make_params(lam, rho, tol, max_iter, precision, k_replace, 8, False, 0)
    items = (BatchItem * len(problems))()
    keep, outs = [], []
    mem = None
    for k, pb in enumerate(problems):
        r = int(pb["r"])
        fb, sizes = _factor_bufs(pb["factors"], r)
        kb, ob, vb = _obs_bufs(pb["kidx"], pb["oidx"], pb["vals"])
        if mem is None:
            mem = kb.mem
        elif kb.mem != mem:
            raise ValueError("every problem of a batch must use the same memory kind")
        n = pb["kernel"].n
        out = pb.get("out")
        if out is None and mem == MEM_HOST:
            out = np.empty((n, r), order="F")
        elif out is None:
            import torch
            out = torch.empty(n * r, dtype=torch.float64, device="cuda")
        wb = _Buf(out, np.float64, colmajor=not _is_torch(out))
        sizes_arr = (ctypes.c_int64 * len(sizes))(*sizes)
        fptrs = (ctypes.c_void_p * len(fb))(*[b.ptr for b in fb])
        flags = (OBS_SORTED if pb.get("sorted_obs") else 0) | _vals_flag(pb["vals"])
        it = items[k]
        it.kern = pb["kernel"].h
        it.d_other = len(fb)
        it.r = r
        it.other_sizes = ctypes.cast(sizes_arr, ctypes.c_void_p)
        it.factors = ctypes.cast(fptrs, ctypes.c_void_p)
        it.q = kb.numel
        it.kidx, it.oidx, it.vals = kb.ptr, ob.ptr, vb.ptr
        it.flags = flags
        it.hold = 1 if pb.get("hold") else 0
        it.W_out = wb.ptr
        keep.append((fb, kb, ob, vb, wb, sizes_arr, fptrs))
        outs.append(wb.obj)
    stats = (Stats * max(1, len(problems)))()
    info = BatchInfo()
    rc = lib().cphifi_solve_batch(ctx.h, len(problems), items, ctypes.byref(prm),
                                  MEM_HOST if mem is None else mem, stats, ctypes.byref(info))
    if rc != OK and info.blocks == 0:  # nothing launched: an argument or creation error
        _check(ctx.h, rc, "solve_batch")
    del keep
    return outs, [stats[k].as_dict() for k in range(len(problems))], info.as_dict()


def gds_noalloc(n: int, r: int, q: int, row_ptr, zhat, ldz: int, Xhat, Y1, stream=None):
    """cphifi_gds_noalloc on device tensors (int64 row_ptr of n + 1 entries,
    FP64 zhat with at least ldz * r entries, FP64 Xhat and Y1 with at least
    n * r entries, all column-major).  Queues the work on `stream` (a
    torch.cuda.Stream, a raw handle or None) and returns without waiting.
    Raises ValueError on a wrong dtype or size, CphifiError on a size beyond
    the entry point's limit or a CUDA failure."""
    import torch
    for t in (row_ptr, zhat, Xhat, Y1):
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise ValueError("gds_noalloc takes contiguous CUDA tensors")
    if row_ptr.dtype != torch.int64:
        raise ValueError("row_ptr must be int64")
    for name, t in (("zhat", zhat), ("Xhat", Xhat), ("Y1", Y1)):
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
    if int(ldz) < int(q):
        raise ValueError("ldz must be >= q")
    if row_ptr.numel() != int(n) + 1:
        raise ValueError("row_ptr must hold n + 1 entries")
    if int(q) > 0 and zhat.numel() < int(ldz) * int(r):
        raise ValueError("zhat must hold ldz * r entries")
    if Xhat.numel() < int(n) * int(r) or Y1.numel() < int(n) * int(r):
        raise ValueError("Xhat and Y1 must hold n * r entries")
    handle = getattr(stream, "cuda_stream", stream) if stream is not None else None
    msg = ctypes.c_char_p()
    rc = lib().cphifi_gds_noalloc(int(n), int(r), int(q), row_ptr.data_ptr(), zhat.data_ptr(),
                                  int(ldz), Xhat.data_ptr(), Y1.data_ptr(),
                                  ctypes.c_void_p(handle), ctypes.byref(msg))
    if rc != OK:
        raise CphifiError(rc, msg.value.decode() if msg.value else status_string(rc))
