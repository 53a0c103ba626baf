"""Plain FP64 CPU oracle of shifted CholeskyQR3.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package. The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``scqr3_oracle.c`` (built with ``-ffp-contract=off`` so
x86-64 and AArch64 give bit-identical results); this module only marshals
numpy arrays into it. ``adjoint.py`` holds the gradient references.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scqr3_oracle.c")
_SO = os.path.join(_HERE, "libscqr3_oracle.so")
MAX_PASSES = 16

OK = 0
E_ARG = -1
E_NONFINITE = -100
E_MAXPASS = -101


def build(force: bool = False) -> str:
    """Compile the oracle into ``libscqr3_oracle.so`` next to its source."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Trace(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int),
                ("shifted", ctypes.c_int * MAX_PASSES),
                ("unshifted_fail", ctypes.c_int * MAX_PASSES),
                ("s", ctypes.c_double * MAX_PASSES),
                ("norm2", ctypes.c_double * MAX_PASSES)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64, i32, f64, p = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.orc_gram.argtypes = [i64, i32, p, i64, p]
        L.orc_gram_oblique.argtypes = [i64, i32, p, i64, i32, p, p, p]
        L.orc_shift.argtypes = [i64, i32, f64]
        L.orc_shift.restype = f64
        L.orc_normest2.argtypes = [i32, p]
        L.orc_normest2.restype = f64
        L.orc_shift_oblique.argtypes = [i64, i32, f64, f64]
        L.orc_shift_oblique.restype = f64
        L.orc_chol.argtypes = [i32, p, f64, p]
        L.orc_chol.restype = i32
        L.orc_trsm.argtypes = [i64, i32, p, i64, p, p, i64]
        L.orc_trmm.argtypes = [i32, p, p]
        L.orc_normb_bound.argtypes = [i64, i32, p]
        L.orc_normb_bound.restype = f64
        L.orc_scqr3.argtypes = [i64, i32, p, i64, i32, p, f64, f64, i32, p, i64, p,
                                ctypes.POINTER(_Trace)]
        L.orc_scqr3.restype = i32
        L.orc_scqr3_ex.argtypes = [i64, i32, p, i64, i32, p, f64, f64, i32, f64, i32, f64, p, i64,
                                   p, ctypes.POINTER(_Trace)]
        L.orc_scqr3_ex.restype = i32
        L.orc_gram_csr.argtypes = [i64, i32, p, i64, p, p, p, p, p]
        L.orc_normb_csr.argtypes = [i64, p, p]
        L.orc_normb_csr.restype = f64
        L.orc_scqr3_csr.argtypes = [i64, i32, p, i64, p, p, p, f64, f64, i32, f64, i32, f64, p,
                                    i64, p, ctypes.POINTER(_Trace)]
        L.orc_scqr3_csr.restype = i32
        _lib = L
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def gram(X: np.ndarray) -> np.ndarray:
    """A = X^T X (Eq. gram)."""
    X = _c(X)
    m, n = X.shape
    A = np.empty((n, n))
    lib().orc_gram(m, n, _ptr(X), n, _ptr(A))
    return A


def gram_oblique(X: np.ndarray, Bblk: np.ndarray):
    """A = X^T (B X) for block-diagonal B given as (m/bs, bs, bs); returns (A, ||X||_F^2)."""
    X = _c(X)
    Bblk = _c(Bblk)
    m, n = X.shape
    bs = Bblk.shape[1]
    A = np.empty((n, n))
    f = ctypes.c_double(0.0)
    lib().orc_gram_oblique(m, n, _ptr(X), n, bs, _ptr(Bblk), _ptr(A), ctypes.byref(f))
    return A, f.value


def shift(m: int, n: int, normx2: float) -> float:
    """s of Eq. (finds2)."""
    return lib().orc_shift(m, n, normx2)


def normest2(A: np.ndarray) -> float:
    """lambda_max of a symmetric positive semidefinite A by the power method
    (the ||Q||_2^2 estimate of the shift, Sec. 4.1)."""
    A = _c(A)
    return lib().orc_normest2(A.shape[0], _ptr(A))


TWO_NORM_EST = -1.0  # normx2 value selecting the power-method estimate of ||Q||_2^2 in every shifted pass


def shift_oblique(m: int, n: int, normx2: float, normb: float) -> float:
    """s of Eq. (finds2B)."""
    return lib().orc_shift_oblique(m, n, normx2, normb)


def chol(A: np.ndarray, s: float = 0.0):
    """(R, fail): R^T R = A + sI, fail = 0 or the 1-based breakdown column."""
    A = _c(A)
    n = A.shape[0]
    R = np.empty((n, n))
    fail = lib().orc_chol(n, _ptr(A), s, _ptr(R))
    return R, fail


def trsm(X: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Q = X R^{-1} by row-wise substitution (Eq. backward2)."""
    X = _c(X)
    R = _c(R)
    m, n = X.shape
    Q = np.empty((m, n))
    lib().orc_trsm(m, n, _ptr(X), n, _ptr(R), _ptr(Q), n)
    return Q


def trmm(Rt: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Rt R for upper triangular operands."""
    Rt = _c(Rt)
    out = _c(R).copy()
    lib().orc_trmm(Rt.shape[0], _ptr(Rt), _ptr(out))
    return out


def _csr(csr):
    row_ptr, col_idx, vals = csr
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col_idx, dtype=np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


def gram_csr(X: np.ndarray, csr):
    """A = X^T (B X) for B given as (row_ptr, col_idx, vals); returns (A, ||X||_F^2)."""
    X = _c(X)
    m, n = X.shape
    rp, ci, v = _csr(csr)
    A = np.empty((n, n))
    f = ctypes.c_double(0.0)
    lib().orc_gram_csr(m, n, _ptr(X), n, _ptr(rp), _ptr(ci), _ptr(v), _ptr(A), ctypes.byref(f))
    return A, f.value


def normb_csr(csr) -> float:
    """Largest absolute row sum of the CSR matrix (>= ||B||_2 for symmetric B)."""
    rp, _, v = _csr(csr)
    return lib().orc_normb_csr(len(rp) - 1, _ptr(rp), _ptr(v))


def normb_bound(Bblk: np.ndarray) -> float:
    Bblk = _c(Bblk)
    nb, bs, _ = Bblk.shape
    return lib().orc_normb_bound(nb * bs, bs, _ptr(Bblk))


def scqr3(X: np.ndarray, Bblk: np.ndarray | None = None, normx2: float = 0.0,
          normb: float = 0.0, max_passes: int = 6, shift_scale: float = 0.0, algorithm: int = 3,
          tol: float = 0.0, csr=None):
    """Shifted CholeskyQR3 (Alg. 3 / Alg. 5 with the breakdown rule of Alg. 2).

    shift_scale = c > 0 first tries the smaller shift c u ||X||^2 of the
    Sec. 6.1 remark (c = 1 is the remark's u ||X||^2), falling back to the safe
    shift of Eq. (finds2) on breakdown; algorithm 2 runs Alg. 2 with its
    orthogonality stopping test (tol <= 0: 6{mn + n(n+1)} u, the bound of
    Thm. maincholqr3). Returns (Q, R, status, trace) where trace is a dict with
    the per-pass record (passes, shifted, unshifted_fail, s, norm2).
    csr = (row_ptr, col_idx, vals) selects a sparse SPD B in CSR form instead
    of the block-diagonal Bblk.
    """
    X = _c(X)
    m, n = X.shape
    Q = np.empty((m, n))
    R = np.empty((n, n))
    tr = _Trace()
    if csr is not None:
        rp, ci, v = _csr(csr)
        if len(rp) != m + 1:
            raise ValueError("row_ptr must have m + 1 entries")
        st = lib().orc_scqr3_csr(m, n, _ptr(X), n, _ptr(rp), _ptr(ci), _ptr(v), normx2, normb,
                                 max_passes, shift_scale, algorithm, tol, _ptr(Q), n, _ptr(R),
                                 ctypes.byref(tr))
        return Q, R, st, _trace_dict(tr)
    if Bblk is None:
        bs, bp = 0, None
    else:
        Bblk = _c(Bblk)
        bs, bp = Bblk.shape[1], _ptr(Bblk)
    st = lib().orc_scqr3_ex(m, n, _ptr(X), n, bs, bp, normx2, normb, max_passes, shift_scale,
                            algorithm, tol, _ptr(Q), n, _ptr(R), ctypes.byref(tr))
    return Q, R, st, _trace_dict(tr)


def _trace_dict(tr):
    k = tr.passes
    return {"passes": k,
            "shifted": list(tr.shifted[:k]),
            "unshifted_fail": list(tr.unshifted_fail[:k]),
            "s": list(tr.s[:k]),
            "norm2": list(tr.norm2[:k])}
