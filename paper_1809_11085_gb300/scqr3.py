"""Python binding of the C ABI in include/scqr3.h (argument marshalling only).

Every step of the factorization runs in libscqr3.so on the GPU; this module
only turns torch tensors into device pointers, sizes the workspace and reads
the per-call record back. There is no CPU fallback: if the library or a GPU
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

MAX_PASSES = 8
MAX_N = 256  # largest n (FP64 and tensor-core forms, B = I); the other forms take n <= 128

OK = 0
E_NONFINITE = -100
E_MAXPASS = -101
E_B_INVALID = -108
E_TIMEOUT = -102
E_CUDA = -103
E_WORKSPACE = -104
E_B_NOT_SPD = -105
E_UNSUPPORTED = -106

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libscqr3.so")


class ScqrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed with status %d" % (what, code))
        self.code = code


class _B(ctypes.Structure):
    _fields_ = [("bs", ctypes.c_int), ("blocks", ctypes.c_void_p), ("norm2", ctypes.c_double),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("nnz", ctypes.c_int64)]


class CsrB:
    """A sparse symmetric positive definite B in CSR form on the device, for the
    oblique inner product (Sec. 5; Sec. 7.2 forms B Q by a sparse product).

    row_ptr: int64 (m + 1,), col_idx: int32 (nnz,), vals: float64 (nnz,), all
    contiguous CUDA tensors. norm2 > 0 gives ||B||_2; otherwise the library
    uses the largest absolute row sum.
    """

    def __init__(self, row_ptr, col_idx, vals, norm2: float = 0.0):
        import torch

        for t, dt, name in ((row_ptr, torch.int64, "row_ptr"), (col_idx, torch.int32, "col_idx"),
                            (vals, torch.float64, "vals")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.dim() == 1
                    and t.is_contiguous()):
                raise TypeError("%s must be a contiguous 1-D %s CUDA tensor" % (name, dt))
        if col_idx.numel() != vals.numel():
            raise ValueError("col_idx and vals must have the same length")
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.m = row_ptr.numel() - 1
        self.nnz = vals.numel()
        self.norm2 = float(norm2)

    @classmethod
    def from_arrays(cls, csr, device="cuda", norm2: float = 0.0):
        """From host (row_ptr, col_idx, vals) arrays (e.g. numpy)."""
        import torch

        rp, ci, v = csr
        return cls(torch.as_tensor(rp, dtype=torch.int64).to(device).contiguous(),
                   torch.as_tensor(ci, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(v, dtype=torch.float64).to(device).contiguous(), norm2)


class _Opts(ctypes.Structure):
    _fields_ = [("max_passes", ctypes.c_int), ("precision", ctypes.c_int),
                ("norm_x2", ctypes.c_double), ("shift_scale", ctypes.c_double),
                ("algorithm", ctypes.c_int), ("tol", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("passes", ctypes.c_int),
                ("shifted", ctypes.c_int * MAX_PASSES),
                ("unshifted_fail", ctypes.c_int * MAX_PASSES),
                ("s", ctypes.c_double * MAX_PASSES),
                ("norm2", ctypes.c_double * MAX_PASSES),
                ("more", ctypes.c_int)]


INFO_BYTES = ctypes.sizeof(_Info)

KERNEL_GRAM, KERNEL_PASS, KERNEL_REDUCE, KERNEL_CHOL, KERNEL_BFACTOR = 0, 1, 2, 3, 4
KERNEL_TCUPDATE = 7
KERNEL_NAMES = {0: "pass_kernel(gram)", 1: "pass_kernel(solve+gram)", 2: "reduce_kernel",
                3: "chol_kernel", 4: "bfactor_kernel", 5: "trsm256_kernel", 6: "df_finish_kernel",
                7: "tc_update_kernel"}


class _LaunchTime(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("pass_", ctypes.c_int), ("ms", ctypes.c_float)]


@dataclass
class Info:
    status: int
    passes: int
    shifted: list = field(default_factory=list)
    unshifted_fail: list = field(default_factory=list)
    s: list = field(default_factory=list)
    norm2: list = field(default_factory=list)
    more: int = 0

    @staticmethod
    def from_bytes(buf: bytes) -> "Info":
        c = _Info.from_buffer_copy(buf)
        k = max(0, min(c.passes, MAX_PASSES))
        return Info(c.status, c.passes, list(c.shifted[:k]), list(c.unshifted_fail[:k]),
                    list(c.s[:k]), list(c.norm2[:k]), c.more)


_lib = None


def lib():
    """Load libscqr3.so (built by paper_1809_11085_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libscqr3.so is not built; run paper_1809_11085_gb300.build.build()")
        L = ctypes.CDLL(_LIB_PATH)
        i64, i32, p, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
        L.scqr3_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(_B), ctypes.POINTER(_Opts),
                                            ctypes.POINTER(sz)]
        L.scqr3_workspace_bytes.restype = i32
        L.scqr3_factor.argtypes = [p, i64, i32, i64, ctypes.POINTER(_B), p, i64, p, p, p, sz,
                                   ctypes.POINTER(_Opts), p, p]
        L.scqr3_factor.restype = i32
        L.scqr3_host_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(_B), ctypes.POINTER(_Opts),
                                                 ctypes.POINTER(sz)]
        L.scqr3_host_workspace_bytes.restype = i32
        L.scqr3_factor_host.argtypes = [p, i64, i32, i64, ctypes.POINTER(_B), p, i64, p, p, p, sz,
                                        ctypes.POINTER(_Opts), p, p]
        L.scqr3_factor_host.restype = i32
        L.scqr3_backward_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(sz)]
        L.scqr3_backward_workspace_bytes.restype = i32
        L.scqr3_backward.argtypes = [p, i64, i32, i64, p, i32, p, i64, p, p, i64, p, sz, p]
        L.scqr3_backward.restype = i32
        L.scqr3_backward_workspace_bytes_ex.argtypes = [i64, i32, ctypes.POINTER(_Opts), ctypes.POINTER(sz)]
        L.scqr3_backward_workspace_bytes_ex.restype = i32
        L.scqr3_backward_ex.argtypes = [p, i64, i32, i64, p, i32, p, i64, p, p, i64, ctypes.POINTER(_Opts), p, sz,
                                        p, p]
        L.scqr3_backward_ex.restype = i32
        L.scqr3_shard_sizes.argtypes = [i64, i32, ctypes.POINTER(_B), ctypes.POINTER(_Opts), ctypes.POINTER(sz),
                                        ctypes.POINTER(sz)]
        L.scqr3_shard_sizes.restype = i32
        L.scqr3_gram_partial.argtypes = [p, i64, i32, i64, ctypes.POINTER(_B), p, p, sz, ctypes.POINTER(_Opts), p, p]
        L.scqr3_gram_partial.restype = i32
        L.scqr3_apply_pass.argtypes = [i32, p, i64, p, i64, i32, i64, ctypes.POINTER(_B), p, i64, p, p, p, sz,
                                       ctypes.POINTER(_Opts), p, p]
        L.scqr3_apply_pass.restype = i32
        L.scqr3_debug_set.argtypes = [i32, ctypes.c_longlong]
        L.scqr3_debug_set.restype = i32
        L.scqr3_timing_begin.argtypes = [i32]
        L.scqr3_timing_begin.restype = i32
        L.scqr3_timing_end.argtypes = [ctypes.POINTER(_LaunchTime), i32, ctypes.POINTER(i32)]
        L.scqr3_timing_end.restype = i32
        _lib = L
    return _lib


DEBUG_WAIT_NS = 1       # hand-off wait limit (ns) of the tensor-core kernels; < 0: default
DEBUG_FUSED_SOLVE = 2   # 1: one-sweep tensor-core substitution (16 < n <= 64); 0: separate launches
DEBUG_WAIT_SCOPE = 3    # kernels the wait limit applies to: bit 0 the Gram, bit 1 the substitution


def debug_set(key: int, value: int) -> None:
    """scqr3_debug_set: process-wide test and tuning hooks (see include/scqr3.h)."""
    r = lib().scqr3_debug_set(int(key), int(value))
    if r != OK:
        raise ScqrError(r, "scqr3_debug_set")


def _check_mat(t, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError("%s must be a 2-D float64 CUDA tensor" % name)
    if t.stride(1) != 1:
        raise ValueError("%s must be row-major (stride(1) == 1)" % name)


def _b_struct(B, normb):
    if B is None:
        return None, None
    import torch

    if isinstance(B, CsrB):
        b = _B(0, None, float(normb or B.norm2), ctypes.c_void_p(B.row_ptr.data_ptr()),
               ctypes.c_void_p(B.col_idx.data_ptr()), ctypes.c_void_p(B.vals.data_ptr()), int(B.nnz))
        return b, ctypes.byref(b)

    if not (isinstance(B, torch.Tensor) and B.is_cuda and B.dtype == torch.float64 and B.dim() == 3
            and B.shape[1] == B.shape[2] and B.is_contiguous()):
        raise TypeError("B must be a CsrB or a contiguous (m/bs, bs, bs) float64 CUDA tensor")
    b = _B(int(B.shape[1]), ctypes.c_void_p(B.data_ptr()), float(normb))
    return b, ctypes.byref(b)


PREC_FP64 = 0
PREC_MIXED = 1
PREC_TC = 2  # FP64-accurate: the Gram matrices and the substitution's off-diagonal blocks on the
             # BF16 tensor cores (exact digit split), FP64 diagonal blocks; n <= 256 with B = I, or
             # n <= 128 with B block-diagonal with blocks of 1, 2, 4 or 8 rows
PREC_MIXED_TC = 3  # the mixed form's substitution with the tensor-core Gram matrices
NORM_X2_TWO_EST = -1.0  # norm_x2 value: ||Q||_2^2 of each shifted pass estimated by the power method
ALG_ADAPTIVE = 2  # Alg. 2: shift only on breakdown, stop on the orthogonality test
ALG_SCQR3 = 3     # Alg. 3: shifted pass, then CholeskyQR2


def _opts(max_passes, norm_x2, precision=PREC_FP64, shift_scale=0.0, algorithm=ALG_SCQR3, tol=0.0):
    o = _Opts(int(max_passes), int(precision), float(norm_x2), float(shift_scale), int(algorithm),
              float(tol))
    return o, ctypes.byref(o)


def workspace_bytes(m: int, n: int, B=None, max_passes: int = 0, norm_x2: float = 0.0,
                    normb: float = 0.0) -> int:
    _, bp = _b_struct(B, normb)
    _, op = _opts(max_passes, norm_x2)
    out = ctypes.c_size_t(0)
    r = lib().scqr3_workspace_bytes(int(m), int(n), bp, op, ctypes.byref(out))
    if r != OK:
        raise ScqrError(r, "scqr3_workspace_bytes")
    return out.value


class Workspace:
    """Reusable device scratch for repeated calls of one shape."""

    def __init__(self, m, n, B=None, max_passes=0, device=None):
        import torch

        self.bytes = workspace_bytes(m, n, B, max_passes)
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.ptr = (base + 255) & ~255
        self.info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=device or "cuda")


def factor(X, B=None, *, max_passes: int = 0, norm_x2: float = 0.0, normb: float = 0.0,
           Q=None, R=None, Rpass=None, workspace: Workspace | None = None, stream=None,
           read_info: bool = True, precision: int = PREC_FP64, shift_scale: float = 0.0,
           algorithm: int = ALG_SCQR3, tol: float = 0.0):
    """Shifted CholeskyQR3 of X (m x n, float64 CUDA tensor) through scqr3_factor.

    Returns (Q, R, info). Q may be passed as X for an in-place factorization.
    shift_scale, algorithm and tol are the scqr3_opts fields of the same names
    (the smaller first shift of the Sec. 6.1 remark; Alg. 2 and its tolerance).
    With read_info=False nothing synchronizes and info is the raw device
    buffer (decode later with Info.from_bytes(buf.cpu().numpy().tobytes())).
    """
    import torch

    _check_mat(X, "X")
    m, n = X.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, device=X.device)
    _check_mat(Q, "Q")
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=X.device)
    if not (R.is_cuda and R.dtype == torch.float64 and R.is_contiguous() and tuple(R.shape) == (n, n)):
        raise TypeError("R must be a contiguous n x n float64 CUDA tensor")
    if Rpass is not None and not (Rpass.is_cuda and Rpass.dtype == torch.float64 and Rpass.is_contiguous()
                                  and Rpass.numel() >= MAX_PASSES * n * n):
        raise TypeError("Rpass must hold MAX_PASSES*n*n float64 on the device")
    if workspace is None:
        workspace = Workspace(m, n, B, max_passes, device=X.device)
    b, bp = _b_struct(B, normb)
    o, op = _opts(max_passes, norm_x2, precision, shift_scale, algorithm, tol)
    if stream is None:
        stream = torch.cuda.current_stream(X.device).cuda_stream
    r = lib().scqr3_factor(X.data_ptr(), m, n, X.stride(0), bp, Q.data_ptr(), Q.stride(0),
                           R.data_ptr(), Rpass.data_ptr() if Rpass is not None else None,
                           workspace.ptr, workspace.bytes, op, workspace.info.data_ptr(),
                           ctypes.c_void_p(stream))
    if r != OK:
        raise ScqrError(r, "scqr3_factor")
    if not read_info:
        return Q, R, workspace.info
    info = Info.from_bytes(workspace.info.cpu().numpy().tobytes())
    return Q, R, info


class HostWorkspace:
    """Device scratch of scqr3_factor_host for repeated calls of one shape:
    the workspace and the m x n device buffer of the iterates."""

    def __init__(self, m, n, B=None, max_passes=0, precision=PREC_FP64, device=None):
        import torch

        _, bp = _b_struct(B, 0.0)
        _, op = _opts(max_passes, 0.0, precision)
        out = ctypes.c_size_t(0)
        r = lib().scqr3_host_workspace_bytes(int(m), int(n), bp, op, ctypes.byref(out))
        if r != OK:
            raise ScqrError(r, "scqr3_host_workspace_bytes")
        self.bytes = out.value
        dev = device or "cuda"
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=dev)
        self.ptr = (self.buf.data_ptr() + 255) & ~255
        self.Qdev = torch.empty((m, n), dtype=torch.float64, device=dev)


def factor_host(X, B=None, *, Q=None, R=None, workspace: HostWorkspace | None = None, stream=None,
                max_passes: int = 0, norm_x2: float = 0.0, normb: float = 0.0,
                precision: int = PREC_FP64, shift_scale: float = 0.0, algorithm: int = ALG_SCQR3,
                tol: float = 0.0):
    """scqr3_factor_host: X, Q, R host (CPU float64 tensors, pinned for overlap).

    Synchronous; returns (Q, R, info). Q may be X for an in-place factorization.
    """
    import torch

    def host_mat(t, name, shape=None):
        if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float64
                and t.dim() == 2 and t.stride(1) == 1):
            raise TypeError("%s must be a row-major 2-D float64 CPU tensor" % name)
        if shape is not None and tuple(t.shape) != shape:
            raise ValueError("%s must have shape %s" % (name, shape))

    host_mat(X, "X")
    m, n = X.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, pin_memory=X.is_pinned())
    host_mat(Q, "Q", (m, n))
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64)
    host_mat(R, "R", (n, n))
    if not R.is_contiguous():
        raise TypeError("R must be contiguous")
    if workspace is None:
        workspace = HostWorkspace(m, n, B, max_passes, precision)
    b, bp = _b_struct(B, normb)
    o, op = _opts(max_passes, norm_x2, precision, shift_scale, algorithm, tol)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    buf = (ctypes.c_char * INFO_BYTES)()
    r = lib().scqr3_factor_host(X.data_ptr(), m, n, X.stride(0), bp, Q.data_ptr(), Q.stride(0),
                                R.data_ptr(), workspace.Qdev.data_ptr(), workspace.ptr, workspace.bytes, op,
                                ctypes.addressof(buf), ctypes.c_void_p(stream))
    if r != OK:
        raise ScqrError(r, "scqr3_factor_host")
    return Q, R, Info.from_bytes(bytes(buf))


def timing_begin(capacity: int = 4096) -> None:
    """Record the device duration of every kernel the library launches from now on."""
    r = lib().scqr3_timing_begin(int(capacity))
    if r != OK:
        raise ScqrError(r, "scqr3_timing_begin")


def timing_end(capacity: int = 4096):
    """Stop recording; returns (records, launches) with records = [(kernel, pass, ms), ...]."""
    buf = (_LaunchTime * capacity)()
    cnt = ctypes.c_int(0)
    r = lib().scqr3_timing_end(buf, int(capacity), ctypes.byref(cnt))
    if r != OK:
        raise ScqrError(r, "scqr3_timing_end")
    k = min(cnt.value, capacity)
    return [(buf[i].kernel, buf[i].pass_, buf[i].ms) for i in range(k)], cnt.value


# --------------------------------------------------------------------------- adjoint

def backward_workspace_bytes(m: int, n: int, precision: int = PREC_FP64) -> int:
    out = ctypes.c_size_t(0)
    _, op = _opts(0, 0.0, precision)
    r = lib().scqr3_backward_workspace_bytes_ex(int(m), int(n), op, ctypes.byref(out))
    if r != OK:
        raise ScqrError(r, "scqr3_backward_workspace_bytes_ex")
    return out.value


class BackwardWorkspace:
    """Device workspace of the adjoint for (m, n) and a precision (PREC_FP64:
    the FP64 row kernel; PREC_TC: the row work on the tensor cores), with the
    device status word that scqr3_backward_ex writes."""

    def __init__(self, m, n, device=None, precision: int = PREC_FP64):
        import torch

        self.precision = int(precision)
        self.bytes = backward_workspace_bytes(m, n, self.precision)
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) & ~255
        self.status = torch.zeros(1, dtype=torch.int32, device=device or "cuda")

    def last_status(self) -> int:
        """Status of the last adjoint run on this workspace (synchronizes)."""
        return int(self.status.item())


def backward(Q, Rpass, passes: int, dQ, dR=None, *, dX=None, workspace: BackwardWorkspace | None = None,
             stream=None, precision: int | None = None):
    """dL/dX of scqr3_factor given dL/dQ and dL/dR, through scqr3_backward_ex.

    precision: PREC_FP64 or PREC_TC (default: the workspace's, else PREC_FP64).
    """
    import torch

    _check_mat(Q, "Q")
    _check_mat(dQ, "dQ")
    m, n = Q.shape
    if precision is None:
        precision = workspace.precision if workspace is not None else PREC_FP64
    if dX is None:
        dX = torch.empty((m, n), dtype=torch.float64, device=Q.device)
    _check_mat(dX, "dX")
    if dR is not None:
        dR = dR.contiguous()
    if workspace is None:
        workspace = BackwardWorkspace(m, n, device=Q.device, precision=precision)
    elif workspace.precision != precision:
        raise ValueError("the workspace was sized for another precision")
    if stream is None:
        stream = torch.cuda.current_stream(Q.device).cuda_stream
    _, op = _opts(0, 0.0, precision)
    r = lib().scqr3_backward_ex(Q.data_ptr(), m, n, Q.stride(0), Rpass.data_ptr(), int(passes),
                                dQ.data_ptr(), dQ.stride(0), dR.data_ptr() if dR is not None else None,
                                dX.data_ptr(), dX.stride(0), op, workspace.ptr, workspace.bytes,
                                workspace.status.data_ptr(), ctypes.c_void_p(stream))
    if r != OK:
        raise ScqrError(r, "scqr3_backward_ex")
    return dX


def _autograd_function():
    import torch

    class SCQR3(torch.autograd.Function):
        """(Q, R) = shifted CholeskyQR3(X), differentiable; saves Q and the per-pass R_k."""

        @staticmethod
        def forward(ctx, X, max_passes=0, precision=PREC_FP64):
            n = X.shape[1]
            Rpass = torch.zeros((MAX_PASSES, n, n), dtype=torch.float64, device=X.device)
            Q, R, info = factor(X.contiguous(), max_passes=max_passes, Rpass=Rpass, precision=precision)
            if info.status not in (OK, E_MAXPASS):
                raise ScqrError(info.status, "scqr3_factor")
            ctx.passes = info.passes
            ctx.precision = backward_precision(precision)
            ctx.save_for_backward(Q, Rpass)
            ctx.info = info
            return Q, R

        @staticmethod
        def backward(ctx, dQ, dR):
            Q, Rpass = ctx.saved_tensors
            if dQ is None:
                dQ = torch.zeros_like(Q)
            ws = BackwardWorkspace(*Q.shape, device=Q.device, precision=ctx.precision)
            dX = backward(Q, Rpass, ctx.passes, dQ.contiguous(), dR, workspace=ws)
            if ctx.precision != PREC_FP64 and ws.last_status() != OK:
                raise ScqrError(ws.last_status(), "scqr3_backward_ex")
            return dX, None, None

    return SCQR3


_SCQR3 = None


def backward_precision(precision: int) -> int:
    """The adjoint's form for a forward precision: the tensor-core adjoint for
    the FP64-accurate tensor-core form with n <= 128, else the FP64 one."""
    return PREC_TC if precision == PREC_TC else PREC_FP64


def qr(X, max_passes: int = 0, precision: int = PREC_FP64):
    """Differentiable shifted CholeskyQR3: returns (Q, R) with X = QR.

    precision selects the forward form (scqr3_opts.precision); the adjoint
    runs on the tensor cores after the PREC_TC form (n <= 128), else in FP64.
    """
    global _SCQR3
    if _SCQR3 is None:
        _SCQR3 = _autograd_function()
    import torch

    if X.shape[1] > 128 and X.requires_grad and torch.is_grad_enabled():
        raise ScqrError(E_UNSUPPORTED, "the adjoint takes n <= 128")
    return _SCQR3.apply(X, max_passes, precision)


# ----------------------------------------------------------------------------- row-partitioned form

class ShardWorkspace:
    """One rank's device state for the row-partitioned calls: the workspace,
    the Gram vectors G (summed over ranks) and G' (this rank's next share), and
    the per-call record."""

    def __init__(self, m_local, n, B=None, normb=0.0, precision=PREC_FP64, max_passes=0, device=None):
        import torch

        _, bp = _b_struct(B, normb)
        _, op = _opts(max_passes, 0.0, precision)
        wb, gw = ctypes.c_size_t(0), ctypes.c_size_t(0)
        r = lib().scqr3_shard_sizes(int(m_local), int(n), bp, op, ctypes.byref(wb), ctypes.byref(gw))
        if r != OK:
            raise ScqrError(r, "scqr3_shard_sizes")
        dev = device or "cuda"
        self.bytes = wb.value
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=dev)
        self.ptr = (self.buf.data_ptr() + 255) & ~255
        self.G = torch.zeros(gw.value, dtype=torch.float64, device=dev)
        self.G_next = torch.zeros(gw.value, dtype=torch.float64, device=dev)
        self.info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=dev)


def gram_partial(X, ws: ShardWorkspace, B=None, *, normb=0.0, precision=PREC_FP64, max_passes=0,
                 shift_scale=0.0, algorithm=ALG_SCQR3, tol=0.0, stream=None):
    """scqr3_gram_partial: start a row-partitioned factorization on this rank
    and write its rows' share of X^T X (or X^T B X) into ws.G."""
    import torch

    _check_mat(X, "X")
    m, n = X.shape
    b, bp = _b_struct(B, normb)
    o, op = _opts(max_passes, 0.0, precision, shift_scale, algorithm, tol)
    if stream is None:
        stream = torch.cuda.current_stream(X.device).cuda_stream
    r = lib().scqr3_gram_partial(X.data_ptr(), m, n, X.stride(0), bp, ws.G.data_ptr(), ws.ptr, ws.bytes, op,
                                 ws.info.data_ptr(), ctypes.c_void_p(stream))
    if r != OK:
        raise ScqrError(r, "scqr3_gram_partial")


def apply_pass(k, m_global, X, Q, R, ws: ShardWorkspace, B=None, *, normb=0.0, precision=PREC_FP64,
               max_passes=0, shift_scale=0.0, algorithm=ALG_SCQR3, tol=0.0, stream=None):
    """scqr3_apply_pass: pass k on this rank from the summed ws.G; writes
    ws.G_next (this rank's share of the next Gram) when another pass follows."""
    import torch

    _check_mat(X, "X")
    _check_mat(Q, "Q")
    m, n = X.shape
    b, bp = _b_struct(B, normb)
    o, op = _opts(max_passes, 0.0, precision, shift_scale, algorithm, tol)
    if stream is None:
        stream = torch.cuda.current_stream(X.device).cuda_stream
    r = lib().scqr3_apply_pass(int(k), ws.G.data_ptr(), int(m_global), X.data_ptr(), m, n, X.stride(0), bp,
                               Q.data_ptr(), Q.stride(0), R.data_ptr(), ws.G_next.data_ptr(), ws.ptr, ws.bytes,
                               op, ws.info.data_ptr(), ctypes.c_void_p(stream))
    if r != OK:
        raise ScqrError(r, "scqr3_apply_pass")


def factor_sharded(X, m_global, allreduce, B=None, *, normb=0.0, Q=None, R=None, precision=PREC_FP64,
                   max_passes=0, shift_scale=0.0, algorithm=ALG_SCQR3, tol=0.0, workspace=None):
    """This rank's part of a row-partitioned factorization of an m_global x n
    X whose rows [r0, r0 + m_local) are X here. allreduce(t) must replace the
    float64 CUDA tensor t by its sum over the ranks (e.g.
    torch.distributed.all_reduce with NCCL; with gloo, through a CPU copy).
    Every rank takes the same pass decisions from the same sums, so all of
    them make the same number of allreduce calls. Returns (Q_local, R, info)."""
    import torch

    m, n = X.shape
    if Q is None:
        Q = torch.empty_like(X)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=X.device)
    ws = workspace or ShardWorkspace(m, n, B, normb, precision, max_passes, device=X.device)
    kw = dict(normb=normb, precision=precision, max_passes=max_passes, shift_scale=shift_scale,
              algorithm=algorithm, tol=tol)
    gram_partial(X, ws, B, **kw)
    allreduce(ws.G)
    for k in range(max_passes or 6):
        apply_pass(k, m_global, X, Q, R, ws, B, **kw)
        info = Info.from_bytes(ws.info.cpu().numpy().tobytes())
        if not info.more:
            break
        allreduce(ws.G_next)
        ws.G, ws.G_next = ws.G_next, ws.G
    return Q, R, info
