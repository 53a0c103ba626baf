"""Batched shifted CholeskyQR3: binding of scqr3_batch_* / scqr3_factor_batched,
CUDA-graph capture, the tile-shape autotuner and a differentiable wrapper.

Argument marshalling and orchestration only: every step of the factorization
runs in libscqr3.so.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import time

from . import scqr3
from .scqr3 import INFO_BYTES, MAX_PASSES, OK, Info, ScqrError, lib


class _Item(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("Rpass", ctypes.c_void_p), ("info", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int), ("ldx", ctypes.c_int64), ("ldq", ctypes.c_int64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("tile_panels", ctypes.c_int * 4)]


def _bind():
    L = lib()
    if not getattr(L, "_batched_bound", False):
        p, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.scqr3_batch_plan_create.argtypes = [ctypes.POINTER(_Item), i32, p, ctypes.POINTER(_Tuning),
                                              ctypes.POINTER(p), ctypes.POINTER(sz)]
        L.scqr3_batch_plan_create.restype = i32
        L.scqr3_batch_plan_upload.argtypes = [p, p, sz, p]
        L.scqr3_batch_plan_upload.restype = i32
        L.scqr3_factor_batched.argtypes = [p, p]
        L.scqr3_factor_batched.restype = i32
        L.scqr3_batch_plan_destroy.argtypes = [p]
        L.scqr3_batch_plan_destroy.restype = None
        L._batched_bound = True
    return L


def tuning(tile_panels=(0, 0, 0, 0), ctas_per_sm=0):
    """Tile shape: row panels per tile for n padded to 16, 32, 64, 128 (0: default 8)."""
    if isinstance(tile_panels, int):
        tile_panels = (tile_panels,) * 4
    return {"ctas_per_sm": int(ctas_per_sm), "tile_panels": [int(t) for t in tile_panels]}


class BatchedQR:
    """A fixed batch of tall-skinny matrices X_i, factorized together.

    Allocates Q_i, R_i (and the per-pass R_k if keep_rpass) and the workspace,
    builds and uploads the plan; run() queues the whole batch (or replays its
    CUDA graph when graph=True).

    precision = scqr3.PREC_FP64 (default) runs the batched kernels of
    scqr3_factor_batched (persistent tile queues over all matrices, FP64).
    precision = scqr3.PREC_TC (or PREC_MIXED_TC) queues one scqr3_factor call
    per matrix with that precision, in order on the stream and on one shared
    workspace (sized for the largest matrix; the calls follow one another on
    the stream, so they never use it at the same time); with graph=True the
    whole sequence is captured once and replayed as one CUDA graph.
    """

    def __init__(self, Xs, *, tune=None, max_passes: int = 0, keep_rpass: bool = False,
                 in_place: bool = False, graph: bool = False, shift_scale: float = 0.0,
                 algorithm: int = 3, tol: float = 0.0, precision: int = scqr3.PREC_FP64):
        import torch

        self.Xs = list(Xs)
        if not self.Xs:
            raise ValueError("empty batch")
        dev = self.Xs[0].device
        for X in self.Xs:
            scqr3._check_mat(X, "X_i")
        self.count = len(self.Xs)
        self.Qs = [X if in_place else torch.empty_like(X) for X in self.Xs]
        self.Rs = [torch.empty((X.shape[1], X.shape[1]), dtype=torch.float64, device=dev) for X in self.Xs]
        self.Rpass = ([torch.zeros((MAX_PASSES, X.shape[1], X.shape[1]), dtype=torch.float64, device=dev)
                       for X in self.Xs] if keep_rpass else None)
        self.info_buf = torch.zeros((self.count, INFO_BYTES), dtype=torch.uint8, device=dev)
        self.precision = int(precision)
        self._plan = None
        self.graph = None
        if self.precision != scqr3.PREC_FP64:
            # one scqr3_factor call per matrix on one shared workspace
            nbytes = max(scqr3.workspace_bytes(X.shape[0], X.shape[1], None, max_passes) for X in self.Xs)
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
            self._opts = scqr3._Opts(int(max_passes), self.precision, 0.0, float(shift_scale), int(algorithm),
                                     float(tol))
            self._calls = [(X.data_ptr(), X.shape[0], X.shape[1], X.stride(0), None, self.Qs[i].data_ptr(),
                            self.Qs[i].stride(0), self.Rs[i].data_ptr(),
                            self.Rpass[i].data_ptr() if keep_rpass else None, self.ws_ptr, nbytes,
                            ctypes.byref(self._opts), self.info_buf[i].data_ptr())
                           for i, X in enumerate(self.Xs)]
            self.tune = None
            if graph:
                self._launch()  # warm-up (and the library's one-time set-up) outside capture
                torch.cuda.synchronize(dev)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._launch()
                self.graph = g
            return
        items = (_Item * self.count)()
        for i, X in enumerate(self.Xs):
            items[i] = _Item(X.data_ptr(), self.Qs[i].data_ptr(), self.Rs[i].data_ptr(),
                             self.Rpass[i].data_ptr() if keep_rpass else None,
                             self.info_buf[i].data_ptr(), X.shape[0], X.shape[1], X.stride(0),
                             self.Qs[i].stride(0))
        self.tune = tune or tuning()
        t = _Tuning(self.tune["ctas_per_sm"], (ctypes.c_int * 4)(*self.tune["tile_panels"]))
        opts = scqr3._Opts(int(max_passes), 0, 0.0, float(shift_scale), int(algorithm), float(tol))
        L = _bind()
        plan = ctypes.c_void_p()
        nbytes = ctypes.c_size_t(0)
        r = L.scqr3_batch_plan_create(items, self.count, ctypes.byref(opts), ctypes.byref(t),
                                      ctypes.byref(plan), ctypes.byref(nbytes))
        if r != OK:
            raise ScqrError(r, "scqr3_batch_plan_create")
        self._plan = plan
        self.ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.ws.data_ptr() + 255) & ~255
        stream = torch.cuda.current_stream(dev).cuda_stream
        r = L.scqr3_batch_plan_upload(plan, self.ws_ptr, nbytes.value, ctypes.c_void_p(stream))
        if r != OK:
            raise ScqrError(r, "scqr3_batch_plan_upload")
        self.graph = None
        if graph:
            self._launch()  # warm-up outside capture
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._launch()
            self.graph = g

    def _launch(self):
        import torch

        stream = torch.cuda.current_stream(self.Xs[0].device).cuda_stream
        if self.precision != scqr3.PREC_FP64:
            f = lib().scqr3_factor
            for a in self._calls:
                r = f(*a, ctypes.c_void_p(stream))
                if r != OK:
                    raise ScqrError(r, "scqr3_factor")
            return
        r = _bind().scqr3_factor_batched(self._plan, ctypes.c_void_p(stream))
        if r != OK:
            raise ScqrError(r, "scqr3_factor_batched")

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch()
        return self.Qs, self.Rs

    def infos(self):
        raw = self.info_buf.cpu().numpy()
        return [Info.from_bytes(raw[i].tobytes()) for i in range(self.count)]

    def __del__(self):
        plan = getattr(self, "_plan", None)
        if plan:
            try:
                _bind().scqr3_batch_plan_destroy(plan)
            except Exception:
                pass
            self._plan = None


# --------------------------------------------------------------------------- autotuner

def _signature(Xs):
    dims = sorted((int(X.shape[0]) // 1024, int(X.shape[1])) for X in Xs)
    return hashlib.sha1(json.dumps(dims).encode()).hexdigest()[:16]


def _cache_path():
    return os.environ.get("SCQR3_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "scqr3", "batched_tune.json"))


def autotune(Xs, candidates=(2, 4, 8, 16, 32), reps: int = 2, use_cache: bool = True, verbose=False):
    """Pick the tile shape (row panels per tile, per size class) for this batch.

    Times a full batched factorization for each uniform candidate, then
    refines each size class in turn (coordinate descent over the same
    candidates); caches the winner by device name and batch signature.
    Returns (tuning, table of timings in ms).
    """
    import torch

    dev = Xs[0].device
    key = "%s|%s" % (torch.cuda.get_device_name(dev), _signature(Xs))
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
        if key in cache:
            return cache[key]["tuning"], cache[key]["ms"]

    def timed(tp):
        b = BatchedQR(Xs, tune=tuning(tp))
        b.run()
        torch.cuda.synchronize(dev)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record()
            b.run()
            e1.record()
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        del b
        return best

    table = {}
    best_tp, best_ms = None, float("inf")
    for c in candidates:
        ms = timed((c, c, c, c))
        table[str((c, c, c, c))] = ms
        if verbose:
            print("tile_panels", c, "%.2f ms" % ms)
        if ms < best_ms:
            best_tp, best_ms = (c, c, c, c), ms
    present = {16: 0, 32: 1, 64: 2, 128: 3}
    classes = sorted({present[16 if X.shape[1] <= 16 else 32 if X.shape[1] <= 32 else 64 if X.shape[1] <= 64 else 128]
                      for X in Xs})
    for cls in classes:
        for c in candidates:
            tp = list(best_tp)
            if tp[cls] == c:
                continue
            tp[cls] = c
            ms = timed(tuple(tp))
            table[str(tuple(tp))] = ms
            if ms < best_ms:
                best_tp, best_ms = tuple(tp), ms
    result = tuning(best_tp)
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[key] = {"tuning": result, "ms": table, "best_ms": best_ms, "when": time.time()}
            json.dump(cache, open(path, "w"), indent=1)
        except Exception:
            pass
    return result, table


# --------------------------------------------------------------------------- differentiable batch

def qr_batched(Xs, tune=None, precision: int = scqr3.PREC_FP64):
    """Differentiable batched factorization: returns ([Q_i], [R_i]).

    The forward pass is one batched launch sequence (precision as for
    BatchedQR); the backward pass applies the adjoint (scqr3_backward_ex; on
    the tensor cores after the PREC_TC form) to each matrix from its Q_i and
    per-pass R_k, all queued on the stream with one workspace sized for the
    largest matrix.
    """
    import torch

    Xs = list(Xs)
    n = len(Xs)

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, *X):
            b = BatchedQR([x.detach().contiguous() for x in X], tune=tune, keep_rpass=True, precision=precision)
            b.run()
            infos = b.infos()
            for i, inf in enumerate(infos):
                if inf.status not in (scqr3.OK, scqr3.E_MAXPASS):
                    raise ScqrError(inf.status, "batched factorization of matrix %d" % i)
            ctx.passes = [inf.passes for inf in infos]
            ctx.save_for_backward(*b.Qs, *b.Rpass)
            return (*b.Qs, *b.Rs)

        @staticmethod
        def backward(ctx, *grads):
            saved = ctx.saved_tensors
            Qs, Rps = saved[:n], saved[n:]
            dQs, dRs = grads[:n], grads[n:]
            bp = scqr3.backward_precision(precision)
            big = max(range(n), key=lambda i: scqr3.backward_workspace_bytes(*Qs[i].shape, precision=bp))
            ws = scqr3.BackwardWorkspace(*Qs[big].shape, device=Qs[big].device, precision=bp)
            out = []
            for i in range(n):
                dQ = dQs[i] if dQs[i] is not None else torch.zeros_like(Qs[i])
                out.append(scqr3.backward(Qs[i], Rps[i], ctx.passes[i], dQ.contiguous(), dRs[i], workspace=ws))
            if bp != scqr3.PREC_FP64 and ws.last_status() != scqr3.OK:
                raise ScqrError(ws.last_status(), "scqr3_backward_ex")
            return tuple(out)

    res = _Fn.apply(*Xs)
    return list(res[:n]), list(res[n:])
