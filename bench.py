#!/usr/bin/env python3
"""Benchmark of the shifted CholeskyQR3 hot path on GB300.

One step = one FP64 shifted CholeskyQR3 factorization X = QR through the C
ABI (scqr3_factor) of a 16,777,216 x 64 matrix X = U diag(sigma) V^T
(sigma geometric 1 -> 1e-10), X and Q resident in HBM (8.6 GB each, far
larger than the 129 MB L2, so no flush is needed between steps).

Prints one JSON line (rank 0). Also reports:
  * roofline of the dominant kernel (the one-sweep tensor-core substitution
    for the headline form, else pass_kernel), timed live per launch with CUDA
    events recorded by the library on its stream, against the FP64 peak
    derived from unit counts and clocks (152 SMs x 2 DFMA/clk x 2 flop x
    2.07 GHz = 1258.6 GFLOP/s); a cuBLAS DGEMM measurement is given beside it;
  * path: the step time against the design's own floor (its FP64-pipe work
    at the FP64 peak plus its Gram MMAs at the sustained BF16 peak);
  * accuracy at full size: R against the exact R factor of diag(sigma) V^T
    (m-independent), and against the CPU oracle run once on the same X in a
    background thread while the GPU legs run;
  * e2e: the same metric with X copied from pinned host memory and Q, R
    copied back inside every timed step;
  * cpu_baseline: the CPU oracle, as it stands, timed on a bounded sample of
    the workload, one single-threaded factorization per host core at once;
  * kappa_sweep: one timed factorization per kappa of the scale-up sweep.

`--impl reference` times the CPU oracle instead (no GPU), on a bounded
sample per step. With --gpus N > 1 (torchrun) every rank factorizes its own
matrix (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sCQR3 rows/s & % roofline at m×n; mixed/batched vs FP64 at ‖QᵀQ−I‖≤1e-13"
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 1.2586
# DRAM bytes per row of a pass_kernel<64> launch, fused solve+Gram and substitution only, from
# the ncu captures summarised in profiles/pass_kernel_fp64_1048576x64_full.md; valid only for
# that kernel source.
PROFILED_KERNEL_SHA = "b447e14d15d0797f"
PROFILED_BYTES_PER_ROW = 992.3
PROFILED_SOLVE_BYTES_PER_ROW = 968.7
PROFILED_BLOCK_BYTES_PER_ROW = 210.3  # pass_kernel<16> on the first 16-column block of a 64-column X
# ncu DRAM bytes per row of one launch of the tensor-core kernels at 1048576 rows: the one-sweep
# substitution and the Gram at n = 64 (profiles/tc_fused_solve_kernel_*, profiles/tc_gram_kernel_*), the
# update kernel at n = 128, where every launch has 32 columns of Y and of x (profiles/tc_update_kernel_*);
# valid for the sources they were taken on and the n they were taken at.
PROFILED_TC = {"tc_solve": ("9b47d483893e89d6", ("tc_common.cuh", "tc_solve.cu"), 737.7, 128),
               "tc_gram": ("ece5f37e2cc61b88", ("tc_common.cuh", "tc_gram.cu"), 518.8, 64),
               "tc_fused": ("84d8d80f4c9a751a", ("tc_common.cuh", "tc_fused.cu"), 981.0, 64)}


def profiled_tc_traffic(kind, m, n):
    """DRAM bytes of one launch of a tensor-core kernel at n columns, or None."""
    import hashlib

    sha, files, per_row, n_prof = PROFILED_TC[kind]
    if sha is None:
        return None
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1809_11085_gb300", "csrc", f), "rb").read())
    return per_row * m if h.hexdigest()[:16] == sha and n == n_prof else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="scqr3", choices=["scqr3", "reference"])
    ap.add_argument("--m", type=int, default=16777216)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--kappa", type=float, default=1e10)
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed", "tc", "mixed_tc"],
                    help="arithmetic of the timed factorization (fp64: FP64 DFMA throughout; tc: FP64 "
                         "substitution with FP64-accurate Gram matrices from exact digit products on the "
                         "BF16 tensor cores; mixed: FP32 pairs + FP64; auto: tc for n <= 128, else fp64)")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--legs", default="all", choices=["all", "main", "csr", "backward", "none"],
                    help="main: only the headline workload; all: also the other configurations; "
                         "csr: the headline plus the sparse-B leg alone; backward: the headline plus "
                         "the adjoint legs at --m x --n")
    ap.add_argument("--csr-grid", type=int, default=2048,
                    help="side of the 2-D grid whose Laplacian is B in the sparse-B leg (m = side^2)")
    return ap.parse_args()


def profiled_traffic(m, n, solve_only=False, tcs=False):
    """roofline.traffic of a pass_kernel<64> launch (tcs: a pass_kernel<32>
    launch on a 32-column block), or None if the kernel changed since the
    capture or none was taken."""
    import hashlib

    h = hashlib.sha256()
    for f in ("fp64_device.cuh", "fp64_kernels.cu"):
        h.update(open(os.path.join(ROOT, "paper_1809_11085_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()[:16]
    if sha != PROFILED_KERNEL_SHA or n != 64:
        return None
    if tcs:
        return PROFILED_BLOCK_BYTES_PER_ROW * m if PROFILED_BLOCK_BYTES_PER_ROW and tc_block_width(n) == 16 else None
    return (PROFILED_SOLVE_BYTES_PER_ROW if solve_only else PROFILED_BYTES_PER_ROW) * m


def max_over_ranks(ms, dist, device):
    """Slowest rank's time (every rank gets it): the job ends when the last replica does."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def replica_value(m, world, ms):
    """Whole-job rows/s of `world` independent replicas of m rows, timed by the slowest."""
    return world * m / (ms * 1e-3)


def flops_of(m, n, passes):
    """Algorithmic FP64 flops of one factorization that ran `passes` passes:
    each pass is one Gram (n(n+1) flops per row: n(n+1)/2 FMAs) and one
    substitution (n^2 flops per row: n(n-1)/2 FMAs and n multiplications)."""
    return passes * m * (n * (n + 1) + n * n)


def gram_mma_flops(m, n):
    """Flops of the MMAs one tensor-core Gram launch issues: per K step of 16
    rows, six MMAs of M = 128 whose N add up to 1280 (digit planes s, s + 1
    against up to four planes side by side, s = 0, 2, 4, 6), 2 * 128 * 16 flops
    per unit of N; n <= 64 one 64-column block over all rows, 64 < n <= 128
    three blocks (0,0), (1,1), (0,1), each over all rows."""
    ksteps = (m + 63) // 64 * 4 if n <= 64 else 3 * ((m + 31) // 32) * 2
    return ksteps * 1280 * 2 * 128 * 16


def tc_gram_roofline(m, n, ms_list):
    """Tensor-pipe figures of the tensor-core Gram launches: the MMAs it issues
    (gram_mma_flops) against the measured sustained BF16 peak (the kernel runs
    inside a long step)."""
    if not ms_list:
        return None
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    issued = gram_mma_flops(m, n)
    useful = m * 36 * n * n * 2  # the 36 digit pairs with s + t <= 7 of every row's outer product
    t = statistics.median(ms_list) * 1e-3
    return {"bound": "tensor", "kernel": "tc_gram_kernel (+ colmax_kernel in the timing)",
            "achieved": issued / t / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": issued / t / 1e12 / peak,
            "useful_digit_tflops": useful / t / 1e12, "ms_per_gram": statistics.median(ms_list),
            "peak_note": "measured sustained bf16 (MEASURED_PEAKS.json)" if peaks else "fallback",
            "traffic": profiled_tc_traffic("tc_gram", m, n)}


def pass_kernel_flops(m, n, kernel, pass_idx, passes, gram_in_pass=True, block=None):
    """FP64 flops done by one pass_kernel launch (0 when the device skipped it).
    gram_in_pass=False: the Gram matrices run on the tensor cores, the pass
    kernel only solves. block = J: the launch solves the J-th 32-column block
    (tensor-core substitution)."""
    from paper_1809_11085_gb300 import scqr3

    if kernel == scqr3.KERNEL_GRAM:
        return m * n * (n + 1) if gram_in_pass else 0
    if kernel == scqr3.KERNEL_PASS:
        if pass_idx >= passes:
            return 0
        if block is not None:
            bw = tc_block_width(n)
            w = min(bw, n - bw * block)
            return m * w * w
        f = m * n * n
        if pass_idx < passes - 1 and gram_in_pass:
            f += m * n * (n + 1)
        return f
    return 0


def fused_used(prec, n):
    """The library runs the one-sweep substitution for the tensor-core form at 16 < n <= 64."""
    from paper_1809_11085_gb300 import scqr3

    return prec == scqr3.PREC_TC and 16 < n <= 64


def fused_fp64_ops(n):
    """FP64-pipe operations per row of one one-sweep substitution: per 16-column
    diagonal block 120 FMAs + 16 multiplies, plus one subtraction per entry an
    off-diagonal product updates (NP = 32: 16 entries; NP = 64: 4 x 16)."""
    np_ = 32 if n <= 32 else 64
    return (np_ // 16) * (16 * 15 // 2 + 16) + (16 if np_ == 32 else 64)


def exact_r(s, V):
    """R factor (positive diagonal) of diag(s) V^T: the exact R of
    X = U diag(s) V^T for orthonormal U, whatever m (numpy Householder QR of an
    n x n matrix)."""
    import numpy as np

    _, Re = np.linalg.qr(np.diag(s) @ V.T)
    return Re * np.sign(np.diag(Re))[:, None]


def rel_fro(A, B):
    import numpy as np

    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


def tc_solve_used(prec, n):
    from paper_1809_11085_gb300 import scqr3

    return prec == scqr3.PREC_TC and n <= 128


def tc_block_width(n):
    """Diagonal-block width of the tensor-core substitution (the library's choice)."""
    return 16 if n <= 64 else 32


def tc_update_cols(n):
    """(block width, columns updated) of each tensor-core update launch of one pass, in launch order."""
    w = tc_block_width(n)
    nb = (n + w - 1) // w
    return [(w, min(32, n - c0)) for J in range(nb) for c0 in range(w * (J + 1), n, 32)]


def tc_update_roofline(m, n, upd):
    """HBM figures of the tensor-core substitution updates x_K -= y_J R_JK: per
    row a launch reads y_J (k = 16 or 32 values) and x_K (n1 <= 32) and writes
    x_K' (n1), 8 bytes each. upd: (ms, (k, n1)) per launch that did work."""
    if not upd:
        return None
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    tsum = sum(t for t, _ in upd) * 1e-3
    byts_all = sum(m * 8 * (k + 2 * n1) for _, (k, n1) in upd)
    byts = byts_all / len(upd)
    t = tsum / len(upd)
    # per 128-row tile: digit s against planes 0..7-s, N = 32 (8 - s), contraction k
    mma_flops = sum(((m + 127) // 128) * 2 * 128 * 32 * 36 * k for _, (k, _) in upd) / len(upd)
    return {"bound": "hbm", "kernel": "tc_update_kernel", "achieved": byts / t / 1e9, "peak": peak, "unit": "GB/s",
            "frac": byts / t / 1e9 / peak, "bytes_per_launch": byts, "ms_per_launch": t * 1e3,
            "launches_per_pass": len(tc_update_cols(n)),
            "tensor_tflops_issued": mma_flops / t / 1e12,
            "peak_note": "measured HBM copy (MEASURED_PEAKS.json)" if peaks else "fallback",
            "traffic": profiled_tc_traffic("tc_solve", m, n)}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle legs

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rows_per_s(n, kappa, target_s, seed=77, max_rows=1 << 21, cores=None):
    """Time the CPU oracle (as it stands: single-threaded) on the host's cores:
    `cores` factorizations of one sample at once, one per thread (the oracle's
    C call releases the interpreter lock), the sample sized for about target_s
    seconds each. Returns (rows/s over all cores, rows per factorization,
    seconds, passes, cores)."""
    import concurrent.futures

    import oracle
    from paper_1809_11085_gb300.testmat import testmat

    cores = cores or host_cores()
    m0 = 32768
    X = testmat(m0, n, kappa, seed=seed)
    t0 = time.perf_counter()
    oracle.scqr3(X)
    t_small = time.perf_counter() - t0
    rows = int(min(max_rows, max(m0, m0 * target_s / max(t_small, 1e-6))))
    rows = max(n, (rows // 1024) * 1024)
    X = testmat(rows, n, kappa, seed=seed + 1)
    with concurrent.futures.ThreadPoolExecutor(cores) as ex:
        t0 = time.perf_counter()
        res = list(ex.map(lambda _: oracle.scqr3(X), range(cores)))
        t = time.perf_counter() - t0
    return cores * rows / t, rows, t, res[0][3]["passes"], cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    import concurrent.futures

    import oracle
    from paper_1809_11085_gb300.testmat import testmat

    # one step = one single-threaded oracle factorization per host core, all
    # at once, of a row sample sized so that warmup + steps stay within a few
    # minutes
    cores = host_cores()
    per_step = max(2.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    m0 = 32768
    X = testmat(m0, args.n, args.kappa, seed=91)
    t0 = time.perf_counter()
    oracle.scqr3(X)
    t_small = time.perf_counter() - t0
    rows = int(min(1 << 21, max(m0, m0 * per_step / max(t_small, 1e-6))))
    rows = max(args.n, (rows // 1024) * 1024)
    X = testmat(rows, args.n, args.kappa, seed=92)
    with concurrent.futures.ThreadPoolExecutor(cores) as ex:
        step = lambda: list(ex.map(lambda _: oracle.scqr3(X), range(cores)))  # noqa: E731
        for _ in range(args.warmup):
            step()
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            step()
            ts.append(time.perf_counter() - t0)
    t = sum(ts) / len(ts)
    v = cores * rows / t
    sample = ("%d x %d rows of the same U diag(sigma) V^T construction (kappa=%g); each step %d single-threaded "
              "factorizations of it at once, one per host core" % (rows, args.n, args.kappa, cores))
    out = {"metric": METRIC, "value": v, "unit": "rows/s", "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "sCQR3 FP64 on a bounded row sample of the %d x %d workload" % (args.m, args.n),
                      "m_sample": rows, "n": args.n, "kappa": args.kappa, "cores": cores},
           "cpu_baseline": {"value": v, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- GPU leg

def dgemm_tflops(torch, dev):
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_1809_11085_gb300 import build, scqr3
    from paper_1809_11085_gb300.testmat import testmat_torch

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    m, n, kappa = args.m, args.n, args.kappa
    X, sig_t, V_t = testmat_torch(m, n, kappa, seed=1000 + 100 * 1 + rank, device=dev)
    Rex = exact_r(sig_t.cpu().numpy(), V_t.cpu().numpy())
    Q = torch.empty_like(X)
    ws = scqr3.Workspace(m, n, device=dev)
    stream = torch.cuda.current_stream(dev)

    pname = args.precision if args.precision != "auto" else ("tc" if n <= 128 else "fp64")
    prec = {"fp64": scqr3.PREC_FP64, "mixed": scqr3.PREC_MIXED, "tc": scqr3.PREC_TC,
            "mixed_tc": scqr3.PREC_MIXED_TC}[pname]
    for _ in range(args.warmup):
        scqr3.factor(X, Q=Q, workspace=ws, read_info=False, precision=prec)
    torch.cuda.synchronize(dev)
    _, R, info = scqr3.factor(X, Q=Q, workspace=ws, precision=prec)
    assert info.status == 0, info

    # accuracy of the result the timed steps recompute
    G = Q.T @ Q
    G -= torch.eye(n, dtype=torch.float64, device=dev)
    orth = torch.linalg.matrix_norm(G, 2).item()
    resid = (torch.linalg.matrix_norm(X - Q @ R) / torch.linalg.matrix_norm(X)).item()
    del G
    Rh_main = R.cpu().numpy()
    dR_exact = rel_fro(Rh_main, Rex)

    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.4)
    scqr3.timing_begin(64 * args.steps + 64)
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record(stream)
    for _ in range(args.steps):
        scqr3.factor(X, Q=Q, workspace=ws, read_info=False, precision=prec)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    recs, launches = scqr3.timing_end(64 * args.steps + 64)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        ms = max_over_ranks(ms, dist, dev)

    passes = info.passes
    value = replica_value(m, world, ms)
    # dominant kernel: pass_kernel launches that did work
    kflops, kms, kl = 0.0, 0.0, 0
    share = {}
    tc_gram_ms, tc_upd_ms = [], []
    tc_path = prec in (scqr3.PREC_TC, scqr3.PREC_MIXED_TC)
    fused = fused_used(prec, n)
    tcs = tc_solve_used(prec, n) and not fused
    fused_ms = []
    seen = {}  # (kernel, pass) -> records so far in the current factorization
    for kernel, p, t in recs:
        name = scqr3.KERNEL_NAMES.get(kernel, str(kernel))
        block = None
        if kernel == scqr3.KERNEL_CHOL and p == 0:
            seen = {}  # a new factorization begins
        j = seen.get((kernel, p), 0)
        seen[(kernel, p)] = j + 1
        if tc_path and kernel == scqr3.KERNEL_GRAM:
            name = "tc_gram_kernel (+ colmax_kernel)"
            if p <= passes - 1:
                tc_gram_ms.append(t)
        if fused and kernel == scqr3.KERNEL_PASS:
            name = "tc_fused_solve_kernel"
            if p < passes:
                fused_ms.append(t)
        if tcs and kernel == scqr3.KERNEL_PASS:
            block = j % ((n + tc_block_width(n) - 1) // tc_block_width(n))
            name = "pass_kernel<32|16> (FP64 diagonal blocks)"
        if tcs and kernel == scqr3.KERNEL_TCUPDATE:
            ucols = tc_update_cols(n)
            jj = j % (len(ucols) + 1)
            name = "tc_update_kernel" if jj > 0 else "tc_split_r_kernel"
            if jj > 0 and p < passes:
                tc_upd_ms.append((t, ucols[jj - 1]))
        share[name] = share.get(name, 0.0) + t
        if fused:
            # DFMA-equivalent flops of the FP64-pipe operations the one-sweep substitution issues
            f = 2 * fused_fp64_ops(n) * m if (kernel == scqr3.KERNEL_PASS and p < passes) else 0
        else:
            f = pass_kernel_flops(m, n, kernel, p, passes,
                                  gram_in_pass=prec not in (scqr3.PREC_TC, scqr3.PREC_MIXED_TC), block=block)
        if f > 0:
            kflops += f
            kms += t
            kl += 1
    tot = sum(share.values()) or 1.0
    achieved = kflops / (kms * 1e-3) / 1e12 if kms > 0 else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    dgemm = dgemm_tflops(torch, dev)

    # the other forms on the same X, one step each (after a warm-up)
    forms = {}
    form_R = {pname: Rh_main}
    if args.legs != "none":
        Rref = R.clone()
        for fname, fp in (("fp64", scqr3.PREC_FP64), ("tc", scqr3.PREC_TC), ("mixed", scqr3.PREC_MIXED),
                          ("mixed_tc", scqr3.PREC_MIXED_TC)):
            if fp == prec or (n > 128 and fp in (scqr3.PREC_TC, scqr3.PREC_MIXED_TC)):
                continue
            fms = _time(torch, stream, lambda: scqr3.factor(X, Q=Q, workspace=ws, read_info=False, precision=fp),
                        reps=2)
            _, Rf, finf = scqr3.factor(X, Q=Q, workspace=ws, precision=fp)
            form_R[fname] = Rf.cpu().numpy()
            forms[fname] = {"ms": round(fms, 2), "rows_per_s": m / (fms * 1e-3), "passes": finf.passes,
                            "orth": _orth(torch, Q),
                            "resid": (torch.linalg.matrix_norm(X - Q @ Rf) / torch.linalg.matrix_norm(X)).item(),
                            "dR_vs_headline": (torch.linalg.matrix_norm(Rf - Rref) /
                                               torch.linalg.matrix_norm(Rref)).item(),
                            "dR_vs_exact": rel_fro(form_R[fname], Rex)}
        # restore the headline's Q for nothing else: the e2e leg has its own buffers

    cpu = None
    if not args.no_cpu:
        v, rows, t, p, cores = oracle_rows_per_s(n, kappa, args.cpu_seconds)
        cpu = {"value": v, "unit": "rows/s", "cores": cores, "kind": "oracle",
               "sample": "%d x %d X = U diag(sigma) V^T, kappa=%g; %d single-threaded factorizations (%d passes) "
                         "at once, one per host core, in %.1f s" % (rows, n, kappa, cores, p, t)}

    # the CPU oracle on the headline X itself, once, in a background thread
    # (its C call releases the interpreter lock) while the other legs run
    oracle_job = None
    if not args.no_cpu:
        import threading

        import oracle

        Xnp = X.cpu().numpy()
        oracle_job = {"t0": time.perf_counter()}

        def _run_oracle():
            try:
                _, Ro, st, tr = oracle.scqr3(Xnp)
                oracle_job.update(R=Ro, status=st, passes=tr["passes"], s=time.perf_counter() - oracle_job["t0"])
            except Exception as exc:  # reported in the line, never fatal to the GPU legs
                oracle_job["error"] = repr(exc)

        oracle_job["thread"] = threading.Thread(target=_run_oracle, daemon=True)
        oracle_job["thread"].start()

    # e2e: pinned host X -> device, factorization, Q and R -> pinned host, every step
    e2e = None
    if not args.no_e2e:
        # the public host-buffer call: X from pinned host memory, Q, R and info
        # back to it, every step, copies overlapped with the work inside the call
        Xh = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Xh.copy_(X)
        Qh = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        hws = scqr3.HostWorkspace(m, n, precision=prec, device=dev)
        ksteps = max(2, min(args.steps, 4))
        scqr3.factor_host(Xh, Q=Qh, R=Rh, workspace=hws, precision=prec)  # warm-up
        torch.cuda.synchronize(dev)
        # the pinned-memory link right before the steps (host memory and the
        # CPU-GPU link are shared with the machine's other jobs)
        tl0 = time.perf_counter()
        hws.Qdev.copy_(Xh, non_blocking=True)
        torch.cuda.synchronize(dev)
        tl1 = time.perf_counter()
        Qh.copy_(hws.Qdev, non_blocking=True)
        torch.cuda.synchronize(dev)
        tl2 = time.perf_counter()
        link = {"h2d_gbs": m * n * 8 / (tl1 - tl0) / 1e9, "d2h_gbs": m * n * 8 / (tl2 - tl1) / 1e9}
        f0, f1 = torch.cuda.Event(True), torch.cuda.Event(True)
        t0 = time.perf_counter()
        f0.record(stream)
        step_ms = []
        for _ in range(ksteps):
            ts = time.perf_counter()
            _, _, hinf = scqr3.factor_host(Xh, Q=Qh, R=Rh, workspace=hws, precision=prec)
            step_ms.append(round((time.perf_counter() - ts) * 1e3, 2))
        f1.record(stream)
        torch.cuda.synchronize(dev)
        wall = (time.perf_counter() - t0) * 1e3 / ksteps
        ems = max(f0.elapsed_time(f1) / ksteps, wall)
        Qchk = Qh.to(dev)
        e2e_orth = _orth(torch, Qchk)
        del Qchk
        e2e = {"value": world * m / (ems * 1e-3), "unit": "rows/s", "ms_per_step": ems,
               "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": m * n * 8 + n * n * 8 + scqr3.INFO_BYTES,
               "status": hinf.status, "passes": hinf.passes, "step_ms": step_ms,
               "median_step_ms": statistics.median(step_ms), "link": link,
               "path": "pinned host X -> scqr3_factor_host (row-chunked copies overlapped with the first "
                       "Gram and the last solve) -> pinned host Q, R, info; synchronous call per step",
               "orth": e2e_orth}
        del Xh, Qh, hws

    sweep = {}
    if not args.no_sweep:
        from paper_1809_11085_gb300.testmat import repeated_small_sigma

        del X
        torch.cuda.empty_cache()
        for kk in (1e2, 1e6, 1e10, 1e14, 1e15, "repeated"):
            sig = repeated_small_sigma(n, 8, 1e-14, 1e7) if kk == "repeated" else None
            Xs, sg, Vs = testmat_torch(m, n, 0.0 if sig is not None else kk, seed=1150 + len(sweep),
                                       device=dev, sigma=sig)
            Rex_s = exact_r(sg.cpu().numpy(), Vs.cpu().numpy())
            scqr3.factor(Xs, Q=Q, workspace=ws, read_info=False, precision=prec)
            torch.cuda.synchronize(dev)
            g0, g1 = torch.cuda.Event(True), torch.cuda.Event(True)
            g0.record(stream)
            _, Rs, inf = scqr3.factor(Xs, Q=Q, workspace=ws, read_info=False, precision=prec)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            inf = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
            Gs = Q.T @ Q
            Gs -= torch.eye(n, dtype=torch.float64, device=dev)
            o = torch.linalg.matrix_norm(Gs, 2).item()
            sweep[str(kk)] = {"ms": round(g0.elapsed_time(g1), 2), "passes": inf.passes,
                              "shifted": inf.shifted, "status": inf.status, "orth": o,
                              "dR_vs_exact": rel_fro(Rs.cpu().numpy(), Rex_s)}
            del Xs, Gs
            torch.cuda.empty_cache()

    legs = {}
    if args.legs == "all":
        legs = extra_legs(torch, dev, stream, args)
    elif args.legs == "csr":
        legs = {"oblique_csr": csr_leg(torch, dev, stream, args.csr_grid)}
    elif args.legs == "backward":
        legs = {"backward": backward_leg(torch, dev, stream, m, n)}

    accuracy = {"dR_vs_exact": dR_exact,
                "exact_note": "||R - R_exact||_F / ||R_exact||_F, R_exact = R factor of diag(sigma) V^T "
                              "(exact for X = U diag(sigma) V^T, U orthonormal to ~1e-15), headline form",
                "forms_dR_vs_exact": {k: v.get("dR_vs_exact") for k, v in forms.items()}}
    if oracle_job is not None:
        oracle_job["thread"].join()
    if oracle_job is not None and "R" in oracle_job:
        Ro = oracle_job["R"]
        accuracy.update({"oracle": "CPU oracle on the same %d x %d X (one run, single-threaded, %.0f s, %d passes, "
                                   "status %d)" % (m, n, oracle_job["s"], oracle_job["passes"],
                                                   oracle_job["status"]),
                         "dR_vs_oracle": {k: rel_fro(v, Ro) for k, v in form_R.items()},
                         "oracle_dR_vs_exact": rel_fro(Ro, Rex)})
    elif oracle_job is not None:
        accuracy["oracle"] = "failed: %s" % oracle_job.get("error")

    # the design's floor: its FP64-pipe work at the FP64 peak plus its Gram MMAs
    # at the sustained BF16 peak (the kernels run one after another)
    path = None
    if fused:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
        hbm = peaks.get("hbm_gbs", 6800.0)
        fp64_ms = passes * fused_fp64_ops(n) * m / (FP64_PEAK_DERIVED_TFLOPS * 1e12 / 2) * 1e3
        grams = passes  # the Gram of X and one after each pass but the last
        tensor_ms = grams * gram_mma_flops(m, n) / (bf16 * 1e12) * 1e3
        byts = m * n * 8 * (1 + 2 * passes + (passes - 1) + 1)  # scan of X, each pass r/w, Gram reads
        hbm_ms = byts / (hbm * 1e9) * 1e3
        floor = fp64_ms + tensor_ms
        path = {"floor_ms": floor, "frac": floor / ms, "fp64_pipe_ms": fp64_ms, "gram_tensor_ms": tensor_ms,
                "hbm_ms_overlapped": hbm_ms, "fp64_ops_per_row_per_pass": fused_fp64_ops(n),
                "note": "floor = the substitution's FP64-pipe operations at 1258.6 GFLOP/s (DFMA rate) + the "
                        "tensor-core Gram MMAs (gram_mma_flops) at the measured sustained BF16 peak; HBM time "
                        "(every byte moved once per kernel) overlaps both; per-kernel fractions below",
                "fp64_6mn2_roofline_ms": 6 * m * n * n / (FP64_PEAK_DERIVED_TFLOPS * 1e12) * 1e3}

    fl = flops_of(m, n, passes)
    out = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "dtype_note": {"fp64": "FP64 throughout",
                       "tc": "FP64 Cholesky, accumulation and triangular substitution blocks; the Gram and "
                             "the off-diagonal substitution blocks from exact digit products "
                             "(7-bit integers in BF16, sums below 2^24 in FP32, folded in int64)",
                       "mixed": "FP32 pairs for Gram and substitution, FP64 shift/Cholesky/accumulation",
                       "mixed_tc": "FP32-pair substitution, exact tensor-core Gram"}[pname],
        "config": {"workload": "sCQR3, X = U diag(sigma) V^T, %d x %d, kappa=%g, precision=%s" % (m, n, kappa, pname),
                   "m": m, "n": n, "kappa": kappa, "passes": passes, "shifted": info.shifted,
                   "l2": "inputs (%.1f GB) larger than the 129 MB L2; no flush" % (m * n * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "alu",
                     "kernel": ("tc_fused_solve_kernel (one sweep per pass: FP64 16-column diagonal blocks, "
                                "off-diagonal blocks on the tensor cores; achieved counts its FP64-pipe operations "
                                "as DFMA-equivalent flops, %d per row)" % (2 * fused_fp64_ops(n))) if fused else
                               ("pass_kernel<32|16> (FP64 DFMA substitution of the 32-column diagonal blocks; "
                                "the off-diagonal blocks on the tensor cores)") if tcs else
                               "pass_kernel<64> (FP64 DFMA%s)" % (", substitution only" if tc_path else ""),
                     "achieved": achieved, "peak": FP64_PEAK_DERIVED_TFLOPS, "unit": "TFLOP/s",
                     "frac": (achieved / FP64_PEAK_DERIVED_TFLOPS) if achieved else None,
                     "traffic": (profiled_tc_traffic("tc_fused", m, n) if fused else
                                 profiled_traffic(m, n, solve_only=tc_path, tcs=tcs)), "traffic_note":
                         "DRAM bytes of one %s launch (ncu at 1048576 rows, scaled by rows)"
                         % ("one-sweep substitution" if fused else "32-column diagonal-block" if tcs else
                            "substitution-only" if tc_path else "fused solve+Gram"),
                     "launches_timed": kl,
                     "peak_note": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; cuBLAS DGEMM measured beside it",
                     "cublas_dgemm_tflops": dgemm},
        "precision": pname,
        "roofline_tc_gram": tc_gram_roofline(m, n, tc_gram_ms) if tc_path else None,
        "roofline_tc_update": tc_update_roofline(m, n, tc_upd_ms) if tcs else None,
        "forms": forms,
        "path_tflops": fl / (ms * 1e-3) / 1e12,
        "gflops_6mn2": 6 * m * n * n / (ms * 1e-3) / 1e9,
        "kernel_share": {k: round(v / tot, 4) for k, v in share.items()},
        "path": path,
        "accuracy": accuracy,
        "orth": orth, "resid": resid,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "kappa_sweep": sweep,
        **legs,
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- other configurations

def _time(torch, stream, fn, reps=1):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _orth(torch, Q, BQ=None):
    n = Q.shape[1]
    G = Q.T @ (Q if BQ is None else BQ)
    G -= torch.eye(n, dtype=torch.float64, device=Q.device)
    return torch.linalg.matrix_norm(G, 2).item()


def csr_leg(torch, dev, stream, side):
    """Oblique inner product with a sparse B in CSR form: the shifted 2-D
    Laplacian on a side x side grid (kappa(B) = 1e3), X of side^2 x 128."""
    from paper_1809_11085_gb300 import scqr3
    from paper_1809_11085_gb300.testmat import laplacian_csr, testmat_torch

    mm, nn = side * side, 128
    X, _, _ = testmat_torch(mm, nn, 1e10, seed=1300, device=dev)
    Bc = scqr3.CsrB.from_arrays(laplacian_csr((side, side), 1e3), device=dev)
    Q = torch.empty_like(X)
    ws = scqr3.Workspace(mm, nn, Bc, device=dev)
    ms = _time(torch, stream, lambda: scqr3.factor(X, Bc, Q=Q, workspace=ws, read_info=False))
    inf = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
    scqr3.timing_begin()
    scqr3.factor(X, Bc, Q=Q, workspace=ws, read_info=False)
    recs, _ = scqr3.timing_end()
    gram_ms = [r[2] for r in recs if r[0] == scqr3.KERNEL_GRAM]
    gram_ms = gram_ms[:inf.passes]  # launches after the last needed Gram return at once
    gram_flops = mm * nn * (nn + 1) + 2 * Bc.nnz * nn  # Q^T Y (upper triangle) + Y = B Q
    Bt = torch.sparse_csr_tensor(Bc.row_ptr, Bc.col_idx.to(torch.int64), Bc.vals, size=(mm, mm))
    return {
        "workload": "FP64 sCQR3 in the B inner product, X %d x 128 (kappa 1e10), B sparse CSR: "
                    "shifted 5-point Laplacian, %d x %d grid, kappa(B) 1e3" % (mm, side, side),
        "ms": round(ms, 2), "rows_per_s": mm / (ms * 1e-3), "passes": inf.passes, "status": inf.status,
        "orth_B": _orth(torch, Q, Bt @ Q), "nnz": Bc.nnz,
        "tflops": (inf.passes * (mm * nn * (nn + 1) + 2 * Bc.nnz * nn + mm * nn * nn)) / (ms * 1e-3) / 1e12,
        "csr_gram_ms": [round(t, 2) for t in gram_ms],
        "csr_gram_frac_fp64_peak": [gram_flops / (t * 1e-3) / 1e12 / FP64_PEAK_DERIVED_TFLOPS for t in gram_ms]}


def backward_leg(torch, dev, stream, mm, nn):
    """The adjoint of the mm x nn factorization (kappa 1e10, 3 passes): the FP64
    adjoint and the tensor-core one on the same saved state."""
    from paper_1809_11085_gb300 import scqr3
    from paper_1809_11085_gb300.testmat import testmat_torch

    X, _, _ = testmat_torch(mm, nn, 1e10, seed=1500, device=dev)
    Rpass = torch.zeros((scqr3.MAX_PASSES, nn, nn), dtype=torch.float64, device=dev)
    Q, R, inf = scqr3.factor(X, Rpass=Rpass)
    dQ = torch.randn(X.shape, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(3))
    dR = torch.randn((nn, nn), dtype=torch.float64, device=dev)
    del X
    bws = scqr3.BackwardWorkspace(mm, nn, device=dev)
    dX = torch.empty_like(Q)
    ms = _time(torch, stream, lambda: scqr3.backward(Q, Rpass, inf.passes, dQ, dR, dX=dX, workspace=bws))
    leg = {"workload": "adjoint of the %d x %d factorization (%d passes)" % (mm, nn, inf.passes),
           "ms": round(ms, 2), "rows_per_s": mm / (ms * 1e-3),
           "tflops": inf.passes * mm * 6 * nn * nn / (ms * 1e-3) / 1e12}
    del bws
    torch.cuda.empty_cache()
    if nn <= 128:  # the same adjoint with its row work on the tensor cores
        bwt = scqr3.BackwardWorkspace(mm, nn, device=dev, precision=scqr3.PREC_TC)
        dXt = torch.empty_like(Q)
        mst = _time(torch, stream, lambda: scqr3.backward(Q, Rpass, inf.passes, dQ, dR, dX=dXt, workspace=bwt))
        leg["tc"] = {"ms": round(mst, 2), "rows_per_s": mm / (mst * 1e-3), "speedup": ms / mst,
                     "status": bwt.last_status(),
                     "dX_vs_fp64": (torch.linalg.matrix_norm(dXt - dX) / torch.linalg.matrix_norm(dX)).item()}
    return leg


def extra_legs(torch, dev, stream, args):
    """The other configurations, one factorization timed each (after one warm-up)."""
    from paper_1809_11085_gb300 import batched, scqr3
    from paper_1809_11085_gb300.testmat import (batched_shapes, block_diag_spd_torch,
                                                repeated_small_sigma, testmat_torch)

    legs = {}
    free = lambda: torch.cuda.empty_cache()  # noqa: E731

    # FP64 scale-up at n = 256
    m, n = 1048576, 256
    sweep = {}
    for kk in (1e2, 1e6, 1e10, 1e14, 1e15, "repeated"):
        sig = repeated_small_sigma(n, 8, 1e-14, 1e7) if kk == "repeated" else None
        X, _, _ = testmat_torch(m, n, 0.0 if sig is not None else kk, seed=1250 + len(sweep), device=dev, sigma=sig)
        Q = torch.empty_like(X)
        ws = scqr3.Workspace(m, n, device=dev)
        ms = _time(torch, stream, lambda: scqr3.factor(X, Q=Q, workspace=ws, read_info=False))
        inf = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
        R64 = None
        row = {"ms": round(ms, 2), "rows_per_s": m / (ms * 1e-3), "passes": inf.passes,
               "status": inf.status, "orth": _orth(torch, Q),
               "tflops": flops_of(m, n, inf.passes) / (ms * 1e-3) / 1e12}
        _, R64, _ = scqr3.factor(X, workspace=ws)
        # the FP64-accurate tensor-core form of the same X (n <= 256, B = I)
        mst = _time(torch, stream, lambda: scqr3.factor(X, Q=Q, workspace=ws, precision=scqr3.PREC_TC,
                                                        read_info=False))
        inft = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
        _, Rt, _ = scqr3.factor(X, workspace=ws, precision=scqr3.PREC_TC)
        row["tc"] = {"ms": round(mst, 2), "rows_per_s": m / (mst * 1e-3), "speedup": ms / mst,
                     "passes": inft.passes, "status": inft.status, "orth": _orth(torch, Q),
                     "dR_vs_fp64": float(torch.linalg.norm(Rt - R64) / torch.linalg.norm(R64))}
        sweep[str(kk)] = row
        del X, Q, ws, R64, Rt
        free()
    legs["scaleup_n256"] = {"workload": "sCQR3, X = U diag(sigma) V^T, 1048576 x 256: FP64 and the "
                                        "FP64-accurate tensor-core form (tc)", "kappa": sweep}

    # mixed and tensor-core forms vs FP64 on the same matrices
    mixed = {}
    for (mm, nn, kk) in ((16777216, 64, 1e10), (8388608, 128, 1e4), (8388608, 128, 1e7), (8388608, 128, 1e10)):
        X, _, _ = testmat_torch(mm, nn, kk, seed=1400 + nn, device=dev)
        Q = torch.empty_like(X)
        ws = scqr3.Workspace(mm, nn, device=dev)
        R64 = torch.empty((nn, nn), dtype=torch.float64, device=dev)
        Rf = torch.empty_like(R64)
        t64 = _time(torch, stream, lambda: scqr3.factor(X, Q=Q, R=R64, workspace=ws, read_info=False))
        row = {"fp64_ms": round(t64, 2), "orth_fp64": _orth(torch, Q)}
        for fname, fp in (("mixed", scqr3.PREC_MIXED), ("mixed_tc", scqr3.PREC_MIXED_TC), ("tc", scqr3.PREC_TC)):
            t = _time(torch, stream, lambda: scqr3.factor(X, Q=Q, R=Rf, workspace=ws, read_info=False,
                                                          precision=fp))
            inf = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
            row[fname] = {
                "ms": round(t, 2), "rows_per_s": mm / (t * 1e-3), "speedup_vs_fp64": t64 / t,
                "orth": _orth(torch, Q),
                "resid": (torch.linalg.matrix_norm(X - Q @ Rf) / torch.linalg.matrix_norm(X)).item(),
                "dR_vs_fp64": (torch.linalg.matrix_norm(Rf - R64) / torch.linalg.matrix_norm(R64)).item(),
                "passes": inf.passes, "status": inf.status}
        mixed["%dx%d_kappa%g" % (mm, nn, kk)] = row
        del X, Q, ws
        free()
    legs["mixed"] = {"workload": "same X through precision FP64, MIXED (FP32 pairs + FP64), MIXED_TC (FP32 pairs "
                                 "+ tensor-core Gram) and TC (FP64 substitution + tensor-core Gram)",
                     "results": mixed}

    # oblique inner product, block-diagonal B (8 x 8 blocks G^T G + 0.1 I)
    mm, nn = 4194304, 128
    X, _, _ = testmat_torch(mm, nn, 1e10, seed=1300, device=dev)
    B = block_diag_spd_torch(mm, 8, seed=1301, device=dev)
    Q = torch.empty_like(X)
    ws = scqr3.Workspace(mm, nn, B, device=dev)
    ms = _time(torch, stream, lambda: scqr3.factor(X, B, Q=Q, workspace=ws, read_info=False))
    inf = scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes())
    BQ = torch.matmul(B, Q.view(-1, 8, nn)).view(mm, nn)
    orth_b = _orth(torch, Q, BQ)
    R64 = scqr3.factor(X, B, Q=Q, workspace=ws)[1].clone()
    # the same through the tensor-core form (Gram of Z = L^T Q and the blocked substitution)
    mst = _time(torch, stream, lambda: scqr3.factor(X, B, Q=Q, workspace=ws, read_info=False,
                                                    precision=scqr3.PREC_TC))
    _, Rt, inft = scqr3.factor(X, B, Q=Q, workspace=ws, precision=scqr3.PREC_TC)
    BQ = torch.matmul(B, Q.view(-1, 8, nn)).view(mm, nn)
    legs["oblique"] = {"workload": "FP64 sCQR3 in the B inner product, X 4194304 x 128 (kappa 1e10), "
                                   "B block diagonal 8x8 G^T G + 0.1 I",
                       "ms": round(ms, 2), "rows_per_s": mm / (ms * 1e-3), "passes": inf.passes,
                       "status": inf.status, "orth_B": orth_b,
                       "tc": {"ms": round(mst, 2), "rows_per_s": mm / (mst * 1e-3), "speedup": ms / mst,
                              "passes": inft.passes, "status": inft.status, "orth_B": _orth(torch, Q, BQ),
                              "dR_vs_fp64": (torch.linalg.matrix_norm(Rt - R64) /
                                             torch.linalg.matrix_norm(R64)).item()}}
    del X, B, Q, ws, BQ
    free()

    legs["oblique_csr"] = csr_leg(torch, dev, stream, args.csr_grid)
    free()

    # backward pass at the headline size
    legs["backward"] = backward_leg(torch, dev, stream, 16777216, 64)
    free()

    # batched: 512 uneven matrices, one graph vs 512 single calls
    shapes = batched_shapes(512, seed=5)
    Xs = [testmat_torch(a, b, c, seed=100 + i, device=dev)[0] for i, (a, b, c) in enumerate(shapes)]
    fl = sum(6 * a * b * b for a, b, _ in shapes)
    wss = {}
    Qs = [torch.empty_like(X) for X in Xs]

    def seq():
        for X, Qi in zip(Xs, Qs):
            key = tuple(X.shape)
            if key not in wss:
                wss[key] = scqr3.Workspace(*key, device=dev)
            scqr3.factor(X, Q=Qi, workspace=wss[key], read_info=False)

    tseq = _time(torch, stream, seq)
    del Qs, wss
    free()
    tune, _ = batched.autotune(Xs, candidates=(8, 32), reps=1)
    bq = batched.BatchedQR(Xs, tune=tune, graph=True)
    tb = _time(torch, stream, bq.run)
    infos = bq.infos()
    worst = max(_orth(torch, Q) for Q in bq.Qs)
    Rb = [R.clone() for R in bq.Rs]
    del bq
    free()
    # the FP64-accurate tensor-core form of the same batch: one graph of the
    # per-matrix launch sequences on one shared workspace
    bt = batched.BatchedQR(Xs, graph=True, precision=scqr3.PREC_TC)
    tt = _time(torch, stream, bt.run)
    infos_t = bt.infos()
    worst_t = max(_orth(torch, Q) for Q in bt.Qs)
    dR_t = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(bt.Rs, Rb))
    legs["batched"] = {"workload": "512 X_i, m_i ~ U[2000, 200000], n_i in {16,32,64,128}, log10 kappa_i ~ U[2,12]",
                       "graph_ms": round(tb, 2), "sequential_ms": round(tseq, 2), "speedup": tseq / tb,
                       "tflops_6mn2": fl / (tb * 1e-3) / 1e12, "worst_orth": worst,
                       "all_ok": all(i.status == 0 for i in infos), "tuning": tune,
                       "tc": {"graph_ms": round(tt, 2), "speedup_vs_fp64_graph": tb / tt,
                              "tflops_6mn2": fl / (tt * 1e-3) / 1e12, "worst_orth": worst_t,
                              "worst_dR_vs_fp64": dR_t, "all_ok": all(i.status == 0 for i in infos_t)}}
    del bt, Rb
    free()
    legs["batched"]["backward"] = batched_backward(torch, dev, stream, Xs)
    del Xs
    free()
    return legs


def batched_backward(torch, dev, stream, Xs):
    """The differentiable batch (batched.qr_batched): the backward pass of
    loss = sum_i <W1_i, Q_i> + <W2_i, R_i> (W seeded Gaussian) over all the
    matrices, after the FP64 and after the tensor-core forward (whose adjoint
    runs on the tensor cores); timed from the start of autograd.grad to its end."""
    from paper_1809_11085_gb300 import batched, scqr3

    g = torch.Generator(dev).manual_seed(9)
    W1 = [torch.randn(X.shape, dtype=torch.float64, device=dev, generator=g) for X in Xs]
    W2 = [torch.randn((X.shape[1], X.shape[1]), dtype=torch.float64, device=dev, generator=g) for X in Xs]
    out, grads = {}, {}
    for name, prec, reps in (("fp64", scqr3.PREC_FP64, 1), ("tc", scqr3.PREC_TC, 2)):
        best = float("inf")
        for _ in range(reps):
            Xg = [X.detach().requires_grad_(True) for X in Xs]
            Qs, Rs = batched.qr_batched(Xg, precision=prec)
            loss = sum((a * q).sum() + (b * r).sum() for a, q, b, r in zip(W1, Qs, W2, Rs))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(stream)
            gs = torch.autograd.grad(loss, Xg)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
            del Qs, Rs, loss, Xg
        out[name] = {"ms": round(best, 2)}
        grads[name] = gs
        torch.cuda.empty_cache()
    out["tc"]["speedup"] = out["fp64"]["ms"] / out["tc"]["ms"]
    # both gradients carry the adjoint's O(n kappa u) error (kappa_i up to 1e12 here)
    out["tc"]["worst_grad_vs_fp64"] = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
                                          for a, b in zip(grads["tc"], grads["fp64"]))
    out["workload"] = ("backward of sum_i <W1_i, Q_i> + <W2_i, R_i> over the 512 matrices (autograd.grad: the "
                       "per-matrix adjoints, one workspace, one stream)")
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
