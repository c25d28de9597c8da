#!/usr/bin/env python
"""Benchmark: time-to-eps of the rank-k solve on one GB300 (and N replicas).

A step is one complete lra_solve (lambda_1 estimate, shift, subspace iteration
on (lambda I - X X^T)^-1 with SVRG solves, CholeskyQR2, Rayleigh-Ritz) on a
synthetic planted-spectrum X resident in HBM.  The default workload is the
precision form: exp_two_gaps 8192 x 1048576 stored in BF16 (the headline
value), with the same matrix stored in FP32 timed beside it (key
``f32_companion``) and the request-loop benchmark on a 2000-request Poisson
stream (key ``serve``).

The JSON line reports the mean device time per solve (CUDA events on the
library's stream), the end-to-end time through the C ABI with host buffers,
the roofline of the dominant kernel (from CUDA events around each of its
launches), the SM clocks seen during the timed region, and the FP64 CPU oracle
timed on a bounded sample.

Multi-GPU: replicas only (each rank solves its own copy; no collective on the
data path); the barrier and max-over-ranks timing follow the launch contract.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lra_inputs as L  # noqa: E402

# the metric this benchmark reports (its headline value is the time-to-eps)
METRIC = "time-to-ε=1e-3 & X-pass HBM GB/s (BF16 vs FP32, 1 GB300); serve p50/p99 latency"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lra", "reference"], default="lra")
    ap.add_argument("--workload", default="exp_two_gaps_8192x1048576")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default=None,
                    help="storage of a dense X (default: the workload's own: BF16 for exp_two_gaps, else FP32)")
    ap.add_argument("--companion", default="auto",
                    help="comma-separated storage types (f32, bf16, f16) of the same matrix timed beside the "
                         "headline; auto: f32,f16 for a BF16 headline on a dense workload; none")
    ap.add_argument("--companion-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true", help="leave out the embedded request-loop benchmark")
    ap.add_argument("--shift", choices=["far", "paper"], default="far")
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-outer", type=int, default=2)
    ap.add_argument("--cpu-sample-cols", type=int, default=32768,
                    help="dense X larger than 2^28 entries: the oracle runs on this many columns "
                         "and its time is scaled by n / cols")
    ap.add_argument("--max-outer", type=int, default=0, help="cap on outer iterations (0 = library default)")
    ap.add_argument("--batch", type=int, default=1, help="samples per SVRG inner step (power of two <= 16)")
    ap.add_argument("--acc", action="store_true", help="accelerated SVRG solves (proximal-point loop)")
    ap.add_argument("--acc-target", type=int, default=0, help="samples per epoch of an accelerated subproblem (0 = n)")
    ap.add_argument("--partition", action="store_true",
                    help="Algorithm 6 with adaptive partitioning and deflation (all branches)")
    ap.add_argument("--serve", action="store_true", help="request-loop benchmark instead")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-mean-ms", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=0,
                    help="worker streams of the request loop (0: the library's default, LRA_SERVE_SLOTS or 8)")
    ap.add_argument("--serve-no-baseline", action="store_true",
                    help="leave out the one-job-at-a-time baseline of the request-loop benchmark")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# environment
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, device) -> float:
    """The largest per-rank value (the job's time is its slowest replica's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def recorded_traffic(workload, storage, kernel):
    """DRAM bytes per launch of `kernel` on `workload` in `storage` from
    profiles/dram_traffic.txt (an ncu capture of the current kernel), or None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if (len(parts) == 4 and not line.startswith("#") and parts[0] == workload and parts[1] == storage
                        and parts[2] == kernel):
                    return int(parts[3])
    except OSError:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.close()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i - 5] for r in rows for i in range(5, 9) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------

def sparse_reference(name):
    """fro2, opt, lambda_k, lambda_{p+1} of a seeded sparse workload, as written
    by tests/golden/make_sparse_opt.py (oracle only)."""
    path = os.path.join(ROOT, "tests", "golden", "zipf_csr_opt.txt")
    with open(path) as f:
        for line in f:
            if line.startswith(name + " "):
                kv = dict(t.split("=") for t in line.split()[1:])
                return {k: float(v) for k, v in kv.items()}
    raise KeyError(f"no reference optimum for {name} in {path}")


def spectrum(wl):
    """(opt, lambda_k, lambda_{p+1}) of a workload: closed form for the planted
    spectra, the stored reference for the sparse ones."""
    if wl.storage == "csr":
        ref = sparse_reference(wl.name)
        return ref["opt"], ref["lambda_k"], ref["lambda_p1"]
    s = wl.sigma()
    return wl.opt(), s[wl.k - 1] ** 2, s[wl.p] ** 2


def theory_rate(wl, lam):
    _, lk, lp1 = spectrum(wl)
    return ((lam - lk) / (lam - lp1)) ** 2


def oracle_sample(wl, Xt_host, args, lam1_hat, outer_sample, threads):
    """Time the FP64 oracle on the same X and seeds: the lambda_1 estimate and
    `outer_sample` outer iterations.  A dense X of more than 2^28 entries (whose
    FP64 copy would not fit the host) is sampled: the oracle runs on its first
    `args.cpu_sample_cols` columns and both times are scaled by n / cols (every
    phase of an outer iteration is linear in n: the X passes, and SVRG epochs
    whose length does not depend on n).  Returns (seconds for the fixed part,
    seconds per outer iteration, the oracle's shift, its E trace, the column
    scale factor)."""
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    from oracle import lra_oracle as O
    scale = 1.0
    if wl.storage != "csr" and wl.d * wl.n > (1 << 28):
        cols = min(wl.n, args.cpu_sample_cols)
        scale = wl.n / cols
        Xt_host = Xt_host[:cols]
        lam1_hat = None
    X64 = O.as64(Xt_host)
    pol = O.SHIFT_FAR if args.shift == "far" else O.SHIFT_PAPER
    _, lk, lp1 = spectrum(wl)
    delta = (lk - lp1) / 1.5 / scale
    t0 = time.perf_counter()
    ctx = O.Context(X64, args.seed, O.Options())
    lh = O.lambda1_estimate(ctx)
    t_fixed = time.perf_counter() - t0
    o = O.Options(shift_policy=pol, delta=delta, min_outer=outer_sample, max_outer=outer_sample,
                  tau={"bf16": 1e-3, "f16": 1e-4}.get(args.storage, 1e-5), batch=args.batch,
                  acc=int(args.acc), acc_target=args.acc_target)
    t0 = time.perf_counter()
    r = O.solve(X64, wl.k, wl.p, args.eps, args.seed, o, lam1_hat=lh)
    t_outer = time.perf_counter() - t0
    del X64
    return t_fixed * scale, t_outer / max(outer_sample, 1) * scale, r.lam, r.E_trace, scale


def oracle_partition(wl, Xt_host, args, delta, threads):
    """Seconds of one full FP64 oracle run of Algorithm 6 (adaptive partitioning
    and deflation) on the same X, seed and Delta."""
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    from oracle import lra_oracle as O
    from oracle import lra_partition as P
    o = O.Options(tau={"bf16": 1e-3, "f16": 1e-4}.get(args.storage, 1e-5), batch=args.batch, acc=int(args.acc),
                  acc_target=args.acc_target)
    t0 = time.perf_counter()
    P.adaptive_solve(O.as64(Xt_host), wl.k, wl.p, args.eps, args.seed, o, delta=delta)
    return time.perf_counter() - t0


def predicted_outer(wl, lam, E_trace, eps):
    """Outer iterations at which the stop rule fires, from the sampled Ritz
    error and the asymptotic rate ((lambda - lambda_k)/(lambda - lambda_{p+1}))^2."""
    opt = spectrum(wl)[0]
    r = theory_rate(wl, lam)
    excess = max(E_trace[-1] - opt, 1e-300)
    target = 0.25 * eps * opt
    extra = max(0.0, math.log(target / excess) / math.log(r)) if excess > target else 0.0
    return len(E_trace) - 1 + int(math.ceil(extra))


def predicted_outer_closed_form(wl, eps):
    """Outer iterations of the FAR shift (lambda = 2 lambda_1 / (1 - 1/4)) from the
    planted spectrum alone: the Ritz error's excess starts near sum_{i<=k} lambda_i
    (a random start) and shrinks by the theory rate per iteration until it is
    (eps/4) opt."""
    s = wl.sigma()
    opt = wl.opt()
    lam = 2.0 * s[0] ** 2 / 0.75
    r = theory_rate(wl, lam)
    excess0 = float(np.sum(s[: wl.k] ** 2))
    return int(math.ceil(math.log(0.25 * eps * opt / excess0) / math.log(r)))


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def make_workload(args, device):
    wl = L.WORKLOADS[args.workload]
    import torch
    Xt, U = L.planted_torch(wl.d, wl.n, wl.sigma(), wl.seed, device=device)
    torch.cuda.synchronize()
    return wl, Xt


class DenseSource:
    """A planted-spectrum dense X (FP32 on the device) and its accounting."""

    tensor = True

    def __init__(self, args, wl, device, lra):
        import torch
        self.wl, self.lra, self.args = wl, lra, args
        self.storage = {"f32": lra.LRA_F32, "bf16": lra.LRA_BF16, "f16": lra.LRA_F16}[args.storage]
        self.esize = 4 if args.storage == "f32" else 2
        self.Xt, Uplant = L.planted_torch(wl.d, wl.n, wl.sigma(), wl.seed, device=device)
        self.Uk = np.ascontiguousarray(Uplant[:, :wl.k])  # the planted top-k directions
        torch.cuda.synchronize()
        self.x_bytes = wl.d * wl.n * self.esize
        self.h2d_bytes = wl.d * wl.n * 4
        self.Xh = None

    def create(self, ctx):
        return self.lra.lra_create_dense(ctx, self.wl.d, self.wl.n, self.lra.LRA_F32, self.Xt, self.wl.d, True,
                                         self.storage)

    def to_host(self):
        import torch
        if self.Xh is None:
            self.Xh = torch.empty(self.Xt.shape, dtype=torch.float32, pin_memory=True)
            self.Xh.copy_(self.Xt)
        return self.Xh

    def drop_device(self):
        self.to_host()
        del self.Xt
        self.Xt = None

    def create_from_host(self, ctx):
        return self.lra.lra_create_dense(ctx, self.wl.d, self.wl.n, self.lra.LRA_F32, self.Xh, self.wl.d, False,
                                         self.storage)

    def err(self, U):
        """||X - U U^T X||_F^2 in FP64, X chunk by chunk of columns."""
        import torch
        Ud = U.double()
        X = self.Xt if self.Xt is not None else self.Xh
        tot, proj = 0.0, 0.0
        for c0 in range(0, X.shape[0], 65536):
            blk = X[c0:c0 + 65536].to(U.device).double()
            tot += float((blk * blk).sum())
            P = blk @ Ud.T
            proj += float((P * P).sum())
            del blk, P
        torch.cuda.empty_cache()
        return tot - proj

    def sin_k(self, U, h=None):
        """sin of the largest principal angle between the span of U's first h
        rows (all k when h is None; rows in Ritz-value order) and the planted
        top-h directions (FP64)."""
        h = self.Uk.shape[1] if h is None else min(h, self.Uk.shape[1])
        Ug = np.linalg.qr(U[:h].double().cpu().numpy().T)[0]
        s = np.linalg.svd(self.Uk[:, :h].T @ Ug, compute_uv=False)
        return float(np.sqrt(max(0.0, 1.0 - float(s.min()) ** 2)))

    def pass_bytes(self, kind, pav, storage=None):
        esize = self.esize if storage is None else (4 if storage == "f32" else 2)
        return self.wl.d * self.wl.n * esize + (self.wl.d + self.wl.n) * pav * 4

    def oracle_input(self, cols=None):
        """The host copy of X (its first `cols` columns when X is sampled)."""
        if self.Xh is None and self.Xt is not None and cols and self.wl.d * self.wl.n > (1 << 28):
            return self.Xt[: min(cols, self.wl.n)].cpu().numpy()
        return self.to_host().numpy()

    def release(self):
        self.Xt = None
        self.Xh = None


class CsrSource:
    """A seeded Zipf CSR X: host arrays, device copies, and its accounting."""

    tensor = False

    def __init__(self, args, wl, device, lra):
        import torch
        self.wl, self.lra, self.args = wl, lra, args
        self.storage = lra.LRA_F32
        self.esize = 4
        self.rowptr, self.colidx, self.val = wl.csr()
        self.nnz = int(self.rowptr[-1])
        self.dev = [torch.from_numpy(a).to(device) for a in (self.rowptr, self.colidx, self.val)]
        self.pinned = None
        self.x_bytes = self.nnz * 8
        self.h2d_bytes = self.rowptr.nbytes + self.colidx.nbytes + self.val.nbytes
        self._sp = None

    def create(self, ctx):
        wl = self.wl
        return self.lra.lra_create_csr(ctx, wl.d, wl.n, self.nnz, *self.dev, True)

    def to_host(self):
        import torch
        if self.pinned is None:
            self.pinned = []
            for a in (self.rowptr, self.colidx, self.val):
                t = torch.empty(a.shape, dtype={np.dtype(np.int64): torch.int64, np.dtype(np.int32): torch.int32,
                                                np.dtype(np.float32): torch.float32}[a.dtype], pin_memory=True)
                t.copy_(torch.from_numpy(a))
                self.pinned.append(t)
        return self.pinned

    def drop_device(self):
        self.to_host()
        self.dev = None

    def create_from_host(self, ctx):
        wl = self.wl
        return self.lra.lra_create_csr(ctx, wl.d, wl.n, self.nnz, *self.pinned, False)

    def xt(self):
        if self._sp is None:
            import scipy.sparse as sp
            self._sp = sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.wl.d, self.wl.n)).T.tocsr()
        return self._sp

    def err(self, U):
        import scipy.sparse  # noqa: F401
        Xt = self.xt()
        Uh = U.double().cpu().numpy().T                       # d x k
        P = np.asarray(Xt.astype(np.float64) @ Uh)
        v = self.val.astype(np.float64)
        return float(np.sum(v * v)) - float(np.sum(P * P))

    def pass_bytes(self, kind, pav, storage=None):
        wl = self.wl
        # compressed index + value of every non-zero, the line pointers, the
        # dense operand and the result (gathers of the operand hit L2)
        if kind == "xtw":
            return self.nnz * 8 + (wl.n + 1) * 8 + (wl.d + wl.n) * pav * 4
        return self.nnz * 8 + (wl.d + 1) * 8 + (wl.n + wl.d) * pav * 4

    def oracle_input(self, cols=None):
        return self.xt()

    def release(self):
        self.dev = None
        self.pinned = None


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch
    wl = L.WORKLOADS[args.workload]
    if wl.storage == "csr":
        import scipy.sparse as sp
        rowptr, colidx, val = wl.csr()
        Xh = sp.csr_matrix((val, colidx, rowptr), shape=(wl.d, wl.n)).T.tocsr()
    else:
        wl, Xt = make_workload(args, f"cuda:{local}")
        if wl.d * wl.n > (1 << 28):
            Xt = Xt[: min(wl.n, args.cpu_sample_cols)]   # the oracle's column sample
        Xh = Xt.cpu().numpy()
        del Xt
        torch.cuda.empty_cache()
    threads = len(os.sched_getaffinity(0))
    lam1 = None
    vals = []
    sample_desc = None
    for i in range(args.warmup + args.steps):
        if args.partition:
            _, lk, lp1 = spectrum(wl)
            v = oracle_partition(wl, Xh, args, (lk - lp1) / 1.5, threads)
            sample_desc = "FP64 oracle's Algorithm 6 on the same X, seed and Delta: one full solve per step"
        else:
            t_fixed, t_outer, lam, E, scale = oracle_sample(wl, Xh, args, lam1, args.cpu_sample_outer, threads)
            if scale > 1.0:
                Lstar = predicted_outer_closed_form(wl, args.eps)
                how = "planted spectrum's theory rate from a random start"
                cols = f" on the first {int(round(wl.n / scale))} of {wl.n} columns, times scaled by n / cols,"
            else:
                Lstar = predicted_outer(wl, lam, E, args.eps)
                how = "sampled Ritz error, theory rate"
                cols = ""
            v = t_fixed + t_outer * Lstar
            sample_desc = (f"FP64 oracle on the same X and seeds{cols} lambda_1 estimate + "
                           f"{args.cpu_sample_outer} outer iterations, extrapolated to {Lstar} outer "
                           f"iterations ({how})")
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "d": wl.d, "n": wl.n, "k": wl.k, "p": wl.p,
                   "storage": "csr" if wl.storage == "csr" else args.storage, "shift": args.shift,
                   "eps": args.eps, "batch": args.batch, "acc": bool(args.acc),
                   "partition": bool(args.partition), "parallelism": "single (rank 0, host cores)"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


KERNEL_NAMES = {("xtw", True): "xtw_tc_kernel", ("xy", True): "xy_tc_kernel",
                ("xtw", False): "spmm_xt_kernel", ("xy", False): "spmm_x_kernel"}


def timed_solves(lra, mat, wl, args, opt, stream, steps, warmup, clocks=None):
    """`warmup` untimed solves, then `steps` solves between two CUDA events on
    the library's stream.  Returns (ms per solve, [(status, report)], U)."""
    import torch
    device = stream.device
    U = torch.zeros(wl.k, wl.d, dtype=torch.float32, device=device)
    ritz = torch.zeros(wl.k, dtype=torch.float64, device=device)
    for _ in range(warmup):
        lra.lra_solve(mat, wl.k, wl.p, args.eps, args.seed, opt, U, ritz, lra.LraReport())
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    reps = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rep = lra.LraReport()
        st = lra.lra_solve(mat, wl.k, wl.p, args.eps, args.seed, opt, U, ritz, rep)
        reps.append((st, rep))
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, reps, U


def kernel_table(reps, src, storage, wl, peaks, peak_kind, workload):
    """Per kernel class: launches, time, algorithmic X-pass GB/s; and the
    roofline object of the dominant class."""
    tot = {"xtw": sum(r.xtw_ms for _, r in reps), "xy": sum(r.xy_ms for _, r in reps),
           "inner": sum(r.inner_ms for _, r in reps)}
    cnt = {"xtw": sum(r.xtw_launches for _, r in reps), "xy": sum(r.xy_launches for _, r in reps),
           "inner": sum(r.inner_launches for _, r in reps)}
    cols = {"xtw": sum(r.xtw_cols for _, r in reps), "xy": sum(r.xy_cols for _, r in reps)}
    per_kernel = {}
    for kk in ("xtw", "xy", "inner"):
        if cnt[kk] > 0:
            e = {"launches": cnt[kk], "ms_total": tot[kk], "ms_per_launch": tot[kk] / cnt[kk]}
            if kk in cols:
                pav = cols[kk] / cnt[kk]
                e["x_pass_gbs"] = src.pass_bytes(kk, pav, storage) / (tot[kk] / cnt[kk] / 1e3) / 1e9
                e["frac_of_hbm"] = e["x_pass_gbs"] / peaks["hbm_gbs"]
            if kk == "inner":
                steps = sum(r.inner_steps for _, r in reps)
                if steps > 0:
                    e["steps"] = steps
                    e["ns_per_step"] = tot[kk] * 1e6 / steps
                    # every CTA of the one-sample loop owns a column group on its
                    # own SM and takes all m steps: steps/s per SM = 1 / step time
                    e["steps_per_s_per_sm"] = 1e9 / e["ns_per_step"]
            per_kernel[kk] = e
    dom = max(tot, key=lambda k: tot[k])
    roof = None
    if dom in ("xtw", "xy") and cnt[dom] > 0:
        pav = cols[dom] / cnt[dom]
        bytes_l = src.pass_bytes(dom, pav, storage)
        t_l = tot[dom] / cnt[dom] / 1e3
        hbm = peaks["hbm_gbs"] * 1e9
        compute_bound = False
        if src.tensor:
            # dense X passes run on tensor cores: BF16 X with 2 BF16 MMAs per
            # k-step (hi/lo small operand), FP32 X as a BF16 pair with 3; the
            # executed tensor flops are compared with the measured sustained BF16 peak
            flops_l = 2.0 * wl.d * wl.n * pav
            mmas = 3 if storage == "f32" else 2
            tens = peaks["bf16_tflops_sustained"] * 1e12 / mmas
            compute_bound = bytes_l / hbm < flops_l / tens
        if compute_bound:
            roof = {"bound": "tensor", "achieved": flops_l / t_l / 1e12, "peak": tens / 1e12,
                    "unit": "TFLOP/s", "frac": flops_l / t_l / tens, "traffic": None}
        else:
            roof = {"bound": "hbm", "achieved": bytes_l / t_l / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": bytes_l / t_l / hbm, "traffic": None}
        kname = KERNEL_NAMES[(dom, src.tensor)]
        roof["traffic"] = recorded_traffic(workload, storage, kname)
        roof.update({"kernel": kname, "launches": cnt[dom], "ms_per_launch": t_l * 1e3,
                     "algorithmic_bytes_per_launch": bytes_l, "x_pass_gbs": bytes_l / t_l / 1e9,
                     "peak_source": peak_kind})
    elif cnt["inner"] > 0:
        roof = {"bound": "latency", "achieved": None, "peak": None, "unit": "steps/s",
                "frac": None, "traffic": None,
                "kernel": "inner_csc_kernel" if wl.storage == "csr" else "svrg_inner1_kernel"}
    return roof, per_kernel, tot


def run_lra(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    import paper_1607_02925_gb300 as lra

    wl = L.WORKLOADS[args.workload]
    src = (CsrSource if wl.storage == "csr" else DenseSource)(args, wl, device, lra)
    storage_name = "csr" if wl.storage == "csr" else args.storage
    opt_val, lk, lp1 = spectrum(wl)
    delta = (lk - lp1) / 1.5
    pol = lra.LRA_SHIFT_FAR if args.shift == "far" else lra.LRA_SHIFT_PAPER
    opt = lra.options(shift_policy=pol, delta=delta, profile=1, batch=args.batch, acc=int(args.acc),
                      acc_target=args.acc_target, partition=int(args.partition))
    if args.max_outer > 0:
        opt.max_outer = args.max_outer
    peaks, peak_kind = measured_peaks()

    ctx = lra.lra_init(local)
    mat = src.create(ctx)
    stream = torch.cuda.ExternalStream(lra.lra_ctx_stream(ctx), device=device)

    # ---- headline: the workload in its storage type, X resident in HBM
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ms_step, reps, U = timed_solves(lra, mat, wl, args, opt, stream, args.steps, args.warmup, clocks)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    if world > 1:
        ms_step = max_over_ranks(ms_step, device)
    last = reps[-1][1]
    # accuracy of the last solve, off the clock (FP64 error against the
    # closed-form or stored reference optimum)
    ratio = src.err(U) / opt_val
    sin_k = src.sin_k(U) if hasattr(src, "sin_k") else None
    sin_10 = src.sin_k(U, 10) if hasattr(src, "sin_k") else None
    roof, per_kernel, tot = kernel_table(reps, src, args.storage, wl, peaks, peak_kind, args.workload)
    lra.lra_mat_destroy(mat)
    mat = None
    torch.cuda.empty_cache()

    # ---- companions: the same matrix, seed and eps in other storage types
    comps = args.companion
    if comps == "auto":
        comps = "f32,f16" if (wl.storage != "csr" and args.storage == "bf16") else "none"
    companions = {}
    for comp_storage in ([] if comps == "none" or wl.storage == "csr" or args.companion_steps <= 0
                         else comps.split(",")):
        cst = {"f32": lra.LRA_F32, "bf16": lra.LRA_BF16, "f16": lra.LRA_F16}[comp_storage]
        copt = lra.options(shift_policy=pol, delta=delta, profile=1, batch=args.batch, acc=int(args.acc),
                           acc_target=args.acc_target, partition=int(args.partition))
        if args.max_outer > 0:
            copt.max_outer = args.max_outer
        m2 = lra.lra_create_dense(ctx, wl.d, wl.n, lra.LRA_F32, src.Xt, wl.d, True, cst)
        ms2, reps2, U2 = timed_solves(lra, m2, wl, args, copt, stream, args.companion_steps, 1)
        if world > 1:
            ms2 = max_over_ranks(ms2, device)
        lra.lra_mat_destroy(m2)
        torch.cuda.empty_cache()
        roof2, pk2, _ = kernel_table(reps2, src, comp_storage, wl, peaks, peak_kind, args.workload)
        companions[comp_storage + "_companion"] = {
            "storage": comp_storage, "time_to_eps_s": ms2 / 1e3, "steps": args.companion_steps, "warmup": 1,
            "ratio_err_over_opt": src.err(U2) / opt_val, "outer_iters": reps2[-1][1].outer_iters,
            "status": reps2[-1][0],
            "x_pass_gbs": {k: v.get("x_pass_gbs") for k, v in pk2.items() if "x_pass_gbs" in v},
            "kernels": pk2, "roofline": roof2,
            "headline_over_companion_time": (ms_step / ms2) if ms2 > 0 else None,
        }
        del U2

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        Uh = torch.empty(wl.k, wl.d, dtype=torch.float32, pin_memory=True)
        rh = torch.empty(wl.k, dtype=torch.float64, pin_memory=True)
        src.drop_device()
        torch.cuda.empty_cache()
        times = []
        for _ in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = src.create_from_host(ctx)
            lra.lra_solve(m2, wl.k, wl.p, args.eps, args.seed, opt, Uh, rh, lra.LraReport())
            lra.lra_mat_destroy(m2)
            times.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(times[1:]), "unit": "s", "steps": args.e2e_steps, "warmup": 1,
               "h2d_bytes_per_step": src.h2d_bytes,
               "d2h_bytes_per_step": wl.d * wl.k * 4 + wl.k * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.partition:
        threads = len(os.sched_getaffinity(0))
        t_full = oracle_partition(wl, src.oracle_input(), args, delta, threads)
        cpu = {"value": t_full, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle's Algorithm 6 on the same X, seed and Delta: one full solve"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = len(os.sched_getaffinity(0))
        t_fixed, t_outer, lam, E, scale = oracle_sample(wl, src.oracle_input(args.cpu_sample_cols), args,
                                                        None, args.cpu_sample_outer, threads)
        Lg = last.outer_iters
        cols = (f" on the first {int(round(wl.n / scale))} of {wl.n} columns (times scaled by n / cols)"
                if scale > 1.0 else "")
        cpu = {"value": t_fixed + t_outer * Lg, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": (f"FP64 oracle on the same X and seeds{cols}: lambda_1 estimate ({t_fixed:.1f} s) "
                          f"+ {args.cpu_sample_outer} outer iterations ({t_outer:.2f} s each), "
                          f"extrapolated to the GPU run's {Lg} outer iterations")}
    lra.lra_finalize(ctx)
    src.release()
    torch.cuda.empty_cache()

    serve = None
    if not args.no_serve and world == 1 and args.workload == "exp_two_gaps_8192x1048576" and args.serve_requests > 0:
        try:
            serve = serve_benchmark(args, local)
        except Exception as e:  # noqa: BLE001 - the headline line is still printed
            serve = {"error": repr(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if storage_name == "csr" else args.storage, "data": "synthetic",
            "config": {"workload": args.workload, "d": wl.d, "n": wl.n, "k": wl.k, "p": wl.p,
                       "storage": storage_name, "shift": args.shift, "eps": args.eps, "batch": args.batch,
                       "acc": bool(args.acc), "partition": bool(args.partition),
                       "l2": "inputs larger than L2 (X %.2f GB per pass)" % (src.x_bytes / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy": {"ratio_err_over_opt": ratio, "sin_vs_planted_uk": sin_k,
                         "sin_vs_planted_u10": sin_10, "outer_iters": last.outer_iters,
                         "status": reps[-1][0]},
            "partition_stages": ([[int(last.part_q[t]), "power" if last.part_kind[t] == 1 else "shift"]
                                  for t in range(last.part_stages)] if args.partition else None),
            "roofline": roof,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": int(sum(r.kernel_launches for _, r in reps)),
            "kernel_ms": {k: v / args.steps for k, v in tot.items()},
            "kernels": per_kernel,
            "phases_ms": {name: sum(r.phase_ms[i] for _, r in reps) / args.steps
                          for i, name in enumerate(["xtw", "xy", "inner", "ritz_gram", "eig", "cholqr2",
                                                    "warm_start", "epilogue"])},
            **companions,
            "serve": serve,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def serve_benchmark(args, local):
    """Request-loop benchmark: a Poisson stream of rank-k requests of uneven
    d, n, k and storage type served by lra_submit / lra_poll, against the same
    stream run one job at a time with FP32 storage through lra_solve.  Returns
    the result as a dict (latencies, throughput, bitwise equality and accuracy
    of sampled results)."""
    import threading

    import torch
    import paper_1607_02925_gb300 as lra

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if args.serve_slots > 0:
        os.environ["LRA_SERVE_SLOTS"] = str(args.serve_slots)
    rng = np.random.default_rng(5)
    nreq = args.serve_requests
    arrivals = np.cumsum(rng.exponential(args.serve_mean_ms / 1e3, size=nreq))
    reqs = []
    for j in range(nreq):
        r = np.random.default_rng(5_000_000 + j)
        reqs.append(dict(d=int(r.choice([256, 1024, 4096])), n=int(r.choice([8192, 65536, 262144])),
                         k=int(r.choice([5, 10, 20, 50])), bf16=bool(r.random() < 0.5)))
    # device-resident pool of planted matrices, one per (d, n, k)
    pool = {}
    for d in (256, 1024, 4096):
        for n in (8192, 65536, 262144):
            ks = sorted({q["k"] for q in reqs if q["d"] == d and q["n"] == n})
            if not ks:
                continue
            g = torch.Generator(device=dev)
            g.manual_seed(d * 1000 + n)
            qu, ru = torch.linalg.qr(torch.randn(d, d, generator=g, device=dev))
            qu = qu * torch.sign(torch.diagonal(ru))[None, :]
            qv, rv = torch.linalg.qr(torch.randn(n, d, generator=g, device=dev))
            qv = qv * torch.sign(torch.diagonal(rv))[None, :]
            for k in ks:
                sig = torch.as_tensor(L.sigma_serving(k, d), device=dev, dtype=torch.float32)
                pool[(d, n, k)] = (qv @ (qu * sig[None, :]).T).contiguous()   # (n, d) = X column-major
            del qu, ru, qv, rv
    torch.cuda.synchronize()
    opt = lra.options(shift_policy=lra.LRA_SHIFT_FAR)

    def make(ctx, q, storage):
        X = pool[(q["d"], q["n"], q["k"])]
        return lra.lra_create_dense(ctx, q["d"], q["n"], lra.LRA_F32, X, q["d"], True, storage)

    # ---- served: continuous batching.  A request's matrix is copied to the
    # device when the request arrives, as long as the matrices already resident
    # (queued or running) leave room for it; otherwise the request waits on the
    # host (its latency counts from its arrival either way).
    ctx = lra.lra_init(local)
    free_b, _ = torch.cuda.mem_get_info(local)
    resident_cap = int(0.5 * free_b)

    def mat_bytes(q):
        dpad = (q["d"] + 127) // 128 * 128
        return dpad * q["n"] * (6 if q["bf16"] else 8)    # FP32 copy + BF16 X, or FP32 X + BF16 pair

    t0 = time.perf_counter()
    done_t = [None] * nreq
    results = [None] * nreq
    outstanding = {}
    cond = threading.Condition()
    state = {"resident": 0, "error": None}

    def submitter():
        try:
            for j, q in enumerate(reqs):
                wait = t0 + arrivals[j] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                need = mat_bytes(q)
                with cond:
                    cond.wait_for(lambda: state["resident"] + need <= resident_cap or state["resident"] == 0)
                    state["resident"] += need
                m = make(ctx, q, lra.LRA_BF16 if q["bf16"] else lra.LRA_F32)
                jid = lra.lra_submit(ctx, m, q["k"], 2 * q["k"], args.eps, 1000 + j, opt)
                with cond:
                    outstanding[jid] = (j, m, need)
        except Exception as e:  # noqa: BLE001 - reported in the result line
            with cond:
                state["error"] = repr(e)

    th = threading.Thread(target=submitter)
    th.start()
    finished = 0
    while finished < nreq:
        with cond:
            items = list(outstanding.items())
            failed = state["error"]
        if failed and not items:
            break
        progressed = False
        for jid, (j, m, need) in items:
            q = reqs[j]
            U = torch.empty(q["k"], q["d"], device=dev)
            r = torch.empty(q["k"], dtype=torch.float64, device=dev)
            st = lra.lra_poll(ctx, jid, 0, U, r, allow=(2, 4, 7, 8))
            if st in (7, 8):
                continue
            done_t[j] = time.perf_counter() - t0
            results[j] = (st, U.cpu().numpy(), r.cpu().numpy())
            lra.lra_mat_destroy(m)
            with cond:
                del outstanding[jid]
                state["resident"] -= need
                cond.notify_all()
            finished += 1
            progressed = True
        if not progressed:
            time.sleep(0.0005)
    th.join()
    if state["error"]:
        raise RuntimeError("request submission failed: " + state["error"])
    lat = np.array(done_t) - arrivals
    span = max(done_t) - arrivals[0]
    # sampled results re-run alone must be bitwise equal, and meet the ratio
    # against the planted closed-form optimum
    nchk = min(50, nreq)
    check = list(range(0, nreq, max(1, nreq // nchk)))[:nchk]
    equal = 0
    worst = 0.0
    for j in check:
        q = reqs[j]
        m = make(ctx, q, lra.LRA_BF16 if q["bf16"] else lra.LRA_F32)
        U = torch.empty(q["k"], q["d"], device=dev)
        r = torch.empty(q["k"], dtype=torch.float64, device=dev)
        lra.lra_solve(m, q["k"], 2 * q["k"], args.eps, 1000 + j, opt, U, r)
        lra.lra_mat_destroy(m)
        equal += int(np.array_equal(U.cpu().numpy(), results[j][1]) and np.array_equal(r.cpu().numpy(), results[j][2]))
        X = pool[(q["d"], q["n"], q["k"])].double()
        Um = torch.from_numpy(results[j][1]).to(dev).double()
        P = X @ Um.T
        err = float((X * X).sum()) - float((P * P).sum())
        del X, P
        worst = max(worst, err / L.closed_form_opt(L.sigma_serving(q["k"], q["d"]), q["k"]))
    lra.lra_finalize(ctx)

    # ---- baseline: one job at a time, FP32 storage, same arrival times
    ctx = lra.lra_init(local)
    tb = 0.0
    blat = []
    for j, q in enumerate([] if args.serve_no_baseline else reqs):
        start = max(tb, arrivals[j])
        ts = time.perf_counter()
        m = make(ctx, q, lra.LRA_F32)
        U = torch.empty(q["k"], q["d"], device=dev)
        r = torch.empty(q["k"], dtype=torch.float64, device=dev)
        lra.lra_solve(m, q["k"], 2 * q["k"], args.eps, 1000 + j, opt, U, r)
        lra.lra_mat_destroy(m)
        tb = start + (time.perf_counter() - ts)
        blat.append(tb - arrivals[j])
    lra.lra_finalize(ctx)
    blat = np.array(blat if blat else [float("nan")])
    del pool
    torch.cuda.empty_cache()
    return {
        "metric": "serve_latency", "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "requests": nreq, "mean_interarrival_ms": args.serve_mean_ms,
        "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
        "jobs_per_s": nreq / span, "bitwise_equal_alone": f"{equal}/{len(check)}",
        "max_ratio_err_over_opt_sampled": worst,
        "statuses": sorted({int(r[0]) for r in results}),
        "baseline_one_at_a_time_f32": {"p50": float(np.percentile(blat, 50)),
                                        "p99": float(np.percentile(blat, 99)),
                                        "jobs_per_s": (nreq / (tb - arrivals[0])) if tb > 0 else None},
        "config": {"workload": "planted small-gap spectrum rescaled to k; d in {256,1024,4096}, "
                               "n in {8192,65536,262144}, k in {5,10,20,50}, p = 2k, FP32/BF16 1:1",
                   "shift": "far", "eps": args.eps, "slots": int(os.environ.get("LRA_SERVE_SLOTS", "8"))},
        "data": "synthetic",
    }


def run_serve(args):
    rank, world, local = dist_env()
    print(json.dumps(serve_benchmark(args, local)), flush=True)
    return 0


def main():
    args = parse_args()
    if args.storage is None:
        args.storage = "bf16" if L.WORKLOADS[args.workload].storage == "bf16" else "f32"
    if args.serve:
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_lra(args)


if __name__ == "__main__":
    sys.exit(main())
