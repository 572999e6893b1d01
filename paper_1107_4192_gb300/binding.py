"""ctypes binding of libkfmeg.so (include/kfmeg.h, include/kfmeg_kernels.h).

Argument marshalling only: every step of the filter and smoother runs in the
library's CUDA kernels.  Tensors passed here must be CUDA, contiguous and of
the dtype the C signature names; PyTorch supplies device memory and streams.
If the library has not been built (``paper_1107_4192_gb300.build.build()``)
every entry point raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkfmeg.so")

KF_OK, KF_ERR_ARG, KF_ERR_NOT_PD, KF_ERR_BUDGET, KF_ERR_CUDA, KF_ERR_NUMERIC, KF_ERR_TIMEOUT, \
    KF_ERR_STATE, KF_ERR_UNSUPPORTED = range(9)
KF_F_IDENTITY, KF_F_CSR, KF_F_DENSE = 0, 1, 2
KF_PREC_FP64, KF_PREC_FP32, KF_PREC_MIXED_BF16X3 = 0, 1, 2
KF_SOLVE_FP64, KF_SOLVE_FP32, KF_SOLVE_FP64_TC, KF_SOLVE_FP64_MEAN = 0, 1, 2, 3
KF_COV_SCALAR, KF_COV_DIAG, KF_COV_DENSE = 0, 1, 2
KF_KC_FILTER_UPDATE, KF_KC_INNOVATION, KF_KC_SMOOTH_GEMM, KF_KC_SMOOTH_SOLVE, KF_KC_PREDICT, \
    KF_KC_SOLVE_FACTOR, KF_KC_SOLVE_GAIN, KF_KC_SMOOTH_GEMM_KERNEL, KF_KC_SOLVE_REFINE, \
    KF_KC_REFINE_EXACT_KERNEL = range(10)


class KfDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("m", ctypes.c_int64), ("T", ctypes.c_int64),
                ("f_kind", ctypes.c_int32), ("prec", ctypes.c_int32), ("solve_prec", ctypes.c_int32),
                ("q_kind", ctypes.c_int32), ("r_kind", ctypes.c_int32), ("joseph_every", ctypes.c_int32),
                ("f_nnz", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_uint64),
                ("checkpoint_every", ctypes.c_int32), ("split_terms", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class KfError(RuntimeError):
    def __init__(self, status: int, where: str, fail_step: int = 0):
        self.status = status
        self.fail_step = fail_step
        super().__init__(f"{where}: {strerror(status)} (status {status}, step {fail_step})")


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double

_SIGS = {
    "kf_plan_footprint": (ctypes.c_int, [ctypes.POINTER(KfDesc), ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_I32)]),
    "kf_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(KfDesc)]),
    "kf_filter": (ctypes.c_int, [_P] * 12 + [ctypes.POINTER(_I64)]),
    "fis_smooth": (ctypes.c_int, [_P, _P, _P, _P, _I64, ctypes.POINTER(_I64)]),
    "mne_solve": (ctypes.c_int, [_P, _P, _I32, _P, _I32, _P, _I64, _I64, _I64, _D, _P, _P]),
    "mne_init": (ctypes.c_int, [_P, _P, _I32, _P, _I32, _P, _I64, _I64, _I64, _D, _P, _P, _P, _P]),
    "kf_solve_host": (ctypes.c_int, [_P] * 14 + [ctypes.POINTER(_I64)]),
    "kf_plan_profile": (ctypes.c_int, [_P, _I32]),
    "kf_plan_profile_read": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_D)]),
    "kf_plan_launch_count": (_I64, [_P]),
    "kf_plan_destroy": (None, [_P]),
    "kf_arena_reserve": (ctypes.c_int, [ctypes.c_uint64]),
    "kf_arena_release": (ctypes.c_int, []),
    "kf_arena_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)] * 3),
    "kf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kfx_gemm": (ctypes.c_int, [_I32, _I32, _I32, _I64, _I64, _I64, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
    "kfx_gemm_exact": (ctypes.c_int, [_I32, _I64, _I64, _I64, _D, _P, _I64, _I32, _P, _I64, _I32, _D, _D, _P, _I64,
                                      _P]),
    "kfx_spd_inverse": (ctypes.c_int, [_I32, _I64, _P, _I64, _P, _I64, ctypes.POINTER(_I64), _P]),
    "kfx_tc_wait_limit": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "kfx_posv_right": (ctypes.c_int, [_I32, _I64, _P, _I64, _I64, _P, _I64, ctypes.POINTER(_I64), _P]),
    "kfx_posv_right_static": (ctypes.c_int, [_I32, _I64, _P, _I64, _I64, _P, _I64, ctypes.POINTER(_I64), _P]),
    "kfx_spmm_fpft": (ctypes.c_int, [_I32, _I64, _P, _P, _P, _P, _I64, _P, _I64, _I32, _P, _P]),
    "kfx_split_bf16": (ctypes.c_int, [_I64, _I64, _P, _I64, _P, _P, _I64, _P]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1107_4192_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def strerror(status: int) -> str:
    return lib().kf_strerror(status).decode()


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _f64(t):
    import torch
    if t is not None and t.dtype != torch.float64:
        raise TypeError("expected float64")
    return _ptr(t)


def _i64(t):
    import torch
    if t is not None and t.dtype != torch.int64:
        raise TypeError("expected int64")
    return _ptr(t)


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _check(st: int, where: str, fail_step: int = 0):
    if st != KF_OK:
        raise KfError(st, where, fail_step)


# ------------------------------------------------------------------- plan API

def make_desc(N, m, T, f_kind=KF_F_IDENTITY, prec=KF_PREC_FP64, solve_prec=KF_SOLVE_FP64,
              q_kind=KF_COV_SCALAR, r_kind=KF_COV_SCALAR, joseph_every=0, f_nnz=0,
              mem_budget_bytes=0, checkpoint_every=0, split_terms=0, stream=None) -> KfDesc:
    return KfDesc(N, m, T, f_kind, prec, solve_prec, q_kind, r_kind, joseph_every, f_nnz,
                  mem_budget_bytes, checkpoint_every, split_terms, _stream(stream))


def kf_plan_footprint(desc: KfDesc):
    w, s, c = ctypes.c_uint64(), ctypes.c_uint64(), _I32()
    st = lib().kf_plan_footprint(ctypes.byref(desc), ctypes.byref(w), ctypes.byref(s), ctypes.byref(c))
    return st, w.value, s.value, c.value


def kf_plan(desc: KfDesc) -> int:
    h = _P()
    _check(lib().kf_plan(ctypes.byref(h), ctypes.byref(desc)), "kf_plan")
    return h.value


def kf_plan_destroy(plan: int):
    lib().kf_plan_destroy(plan)


def kf_filter(plan, F, F_rowptr, F_col, Q, H, R, Y, x0, P0, x_filt, diagP_filt=None, raise_on_error=True):
    fs = _I64()
    st = lib().kf_filter(plan, _f64(F), _i64(F_rowptr), _i64(F_col), _f64(Q), _f64(H), _f64(R), _f64(Y),
                         _f64(x0), _f64(P0), _f64(x_filt), _f64(diagP_filt), ctypes.byref(fs))
    if raise_on_error:
        _check(st, "kf_filter", fs.value)
    return st, fs.value


def fis_smooth(plan, x_smooth, diagP_smooth=None, P_smooth_at=None, t_full=-1, raise_on_error=True):
    fs = _I64()
    st = lib().fis_smooth(plan, _f64(x_smooth), _f64(diagP_smooth), _f64(P_smooth_at), t_full, ctypes.byref(fs))
    if raise_on_error:
        _check(st, "fis_smooth", fs.value)
    return st, fs.value


def mne_solve(H, C, c_kind, R, r_kind, Y, N, m, T, lam, X_out, stream=None):
    st = lib().mne_solve(_f64(H), _f64(C), c_kind, _f64(R), r_kind, _f64(Y), N, m, T, lam, _f64(X_out),
                         _stream(stream))
    _check(st, "mne_solve")


def mne_init(H, C, c_kind, R, r_kind, Y, N, m, T, lam, X_out, x0_out, Q_out, stream=None):
    st = lib().mne_init(_f64(H), _f64(C), c_kind, _f64(R), r_kind, _f64(Y), N, m, T, lam,
                        _f64(X_out) if X_out is not None else None, _f64(x0_out), _f64(Q_out),
                        _stream(stream))
    _check(st, "mne_init")


def _hp(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous array")
        return a.ctypes.data
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return a.data_ptr()


def kf_solve_host(plan, F, F_rowptr, F_col, Q, H, R, Y, x0, P0, x_filt, diagP_filt, x_smooth, diagP_smooth):
    """Host buffers in and out (numpy arrays or CPU tensors, pinned for async copies)."""
    fs = _I64()
    st = lib().kf_solve_host(plan, _hp(F), _hp(F_rowptr), _hp(F_col), _hp(Q), _hp(H), _hp(R), _hp(Y), _hp(x0),
                             _hp(P0), _hp(x_filt), _hp(diagP_filt), _hp(x_smooth), _hp(diagP_smooth),
                             ctypes.byref(fs))
    _check(st, "kf_solve_host", fs.value)


def kf_arena_reserve(nbytes: int):
    _check(lib().kf_arena_reserve(int(nbytes)), "kf_arena_reserve")


def kf_arena_release():
    _check(lib().kf_arena_release(), "kf_arena_release")


def kf_arena_stats():
    r, u, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().kf_arena_stats(ctypes.byref(r), ctypes.byref(u), ctypes.byref(f)), "kf_arena_stats")
    return r.value, u.value, f.value


def kf_plan_profile(plan, enable: bool):
    _check(lib().kf_plan_profile(plan, 1 if enable else 0), "kf_plan_profile")


def kf_plan_profile_read(plan, cls: int):
    n, ms = _I64(), _D()
    _check(lib().kf_plan_profile_read(plan, cls, ctypes.byref(n), ctypes.byref(ms)), "kf_plan_profile_read")
    return n.value, ms.value


def kf_plan_launch_count(plan) -> int:
    return lib().kf_plan_launch_count(plan)


# ----------------------------------------------------------- kernel-level API

def kfx_gemm(dtype, transB, sym, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    _check(lib().kfx_gemm(dtype, transB, sym, M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc,
                          _stream(stream)), "kfx_gemm")


def kfx_gemm_exact(levels, M, N, K, alpha, A, lda, B, ldb, beta, delta, C, ldc, stream=None):
    """C = alpha A B^T + beta C + delta I as an exact-slice tensor-core product (float64 C)."""
    import torch
    a32 = 1 if A.dtype == torch.float32 else 0
    b32 = 1 if B.dtype == torch.float32 else 0
    _check(lib().kfx_gemm_exact(levels, M, N, K, alpha, _ptr(A), lda, a32, _ptr(B), ldb, b32, beta, delta, _f64(C),
                                ldc, _stream(stream)), "kfx_gemm_exact")


def kfx_spd_inverse(mode, n, A, lda, X, ldx, stream=None):
    """X = A^{-1} (float32 SPD A, float64 X); mode 1 float32-class, 2 float64-accurate."""
    fi = _I64()
    st = lib().kfx_spd_inverse(mode, n, _ptr(A), lda, _f64(X), ldx, ctypes.byref(fi), _stream(stream))
    return st, fi.value


def kfx_tc_wait_limit(ns: int) -> int:
    """Sets the tensor-core kernels' pipeline-wait limit (0 = default 2 s); returns the old one."""
    prev = ctypes.c_uint64()
    _check(lib().kfx_tc_wait_limit(ns, ctypes.byref(prev)), "kfx_tc_wait_limit")
    return prev.value


def kfx_posv_right(dtype, n, A, lda, M, B, ldb, stream=None):
    fi = _I64()
    st = lib().kfx_posv_right(dtype, n, _ptr(A), lda, M, _ptr(B), ldb, ctypes.byref(fi), _stream(stream))
    return st, fi.value


def kfx_posv_right_static(dtype, n, A, lda, M, B, ldb, stream=None):
    """kfx_posv_right with scratch in a static device array (no allocation); n <= 4096."""
    fi = _I64()
    st = lib().kfx_posv_right_static(dtype, n, _ptr(A), lda, M, _ptr(B), ldb, ctypes.byref(fi), _stream(stream))
    return st, fi.value


def kfx_spmm_fpft(dtype, N, rowptr, col, val, P, ldp, out, ldo, q_kind, Q, stream=None):
    _check(lib().kfx_spmm_fpft(dtype, N, _i64(rowptr), _i64(col), _f64(val), _ptr(P), ldp, _ptr(out), ldo,
                               q_kind, _f64(Q), _stream(stream)), "kfx_spmm_fpft")


def kfx_split_bf16(rows, cols, A, lda, hi, lo, ldh, stream=None):
    _check(lib().kfx_split_bf16(rows, cols, _ptr(A), lda, _ptr(hi), _ptr(lo), ldh, _stream(stream)),
           "kfx_split_bf16")
