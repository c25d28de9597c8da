#!/usr/bin/env python
"""Benchmark: time-to-eps of the rank-k solve on one GB300 (and N replicas).

A step is one complete lra_solve (lambda_1 estimate, shift, subspace iteration
on (lambda I - X X^T)^-1 with SVRG solves, CholeskyQR2, Rayleigh-Ritz) on a
synthetic planted-spectrum X resident in HBM.  The JSON line reports the mean
device time per solve (CUDA events on the library's stream), the end-to-end
time through the C ABI with host buffers, the roofline of the dominant kernel
(from CUDA events around each of its launches), the SM clocks seen during the
timed region, and the FP64 CPU oracle timed on a bounded sample.

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


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lra", "reference"], default="lra")
    ap.add_argument("--workload", default="steep_head_4096x262144")
    ap.add_argument("--storage", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--shift", choices=["far", "paper"], default="far")
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-outer", type=int, default=4)
    ap.add_argument("--max-outer", type=int, default=0, help="cap on outer iterations (0 = library default)")
    ap.add_argument("--batch", type=int, default=1, help="samples per SVRG inner step (power of two <= 16)")
    ap.add_argument("--acc", action="store_true", help="accelerated SVRG solves (proximal-point loop)")
    ap.add_argument("--acc-target", type=int, default=0, help="samples per epoch of an accelerated subproblem (0 = n)")
    ap.add_argument("--partition", action="store_true",
                    help="Algorithm 6 with adaptive partitioning and deflation (all branches)")
    ap.add_argument("--serve", action="store_true", help="request-loop benchmark instead")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-mean-ms", type=float, default=20.0)
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


def recorded_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` on `workload` from profiles/dram_traffic.txt
    (an ncu capture of the current kernel), or None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and not line.startswith("#") and parts[0] == workload and parts[1] == kernel:
                    return int(parts[2])
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
    `outer_sample` outer iterations; returns (seconds for the fixed part,
    seconds per outer iteration, the oracle's shift, its E trace)."""
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    from oracle import lra_oracle as O
    X64 = O.as64(Xt_host)
    pol = O.SHIFT_FAR if args.shift == "far" else O.SHIFT_PAPER
    _, lk, lp1 = spectrum(wl)
    delta = (lk - lp1) / 1.5
    t0 = time.perf_counter()
    ctx = O.Context(X64, args.seed, O.Options())
    lh = O.lambda1_estimate(ctx)
    t_fixed = time.perf_counter() - t0
    o = O.Options(shift_policy=pol, delta=delta, min_outer=outer_sample, max_outer=outer_sample,
                  tau=1e-3 if args.storage == "bf16" else 1e-5, batch=args.batch,
                  acc=int(args.acc), acc_target=args.acc_target)
    t0 = time.perf_counter()
    r = O.solve(X64, wl.k, wl.p, args.eps, args.seed, o, lam1_hat=lh)
    t_outer = time.perf_counter() - t0
    return t_fixed, t_outer / max(outer_sample, 1), r.lam, r.E_trace


def oracle_partition(wl, Xt_host, args, delta, threads):
    """Seconds of one full FP64 oracle run of Algorithm 6 (adaptive partitioning
    and deflation) on the same X, seed and Delta."""
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    from oracle import lra_oracle as O
    from oracle import lra_partition as P
    o = O.Options(tau=1e-3 if args.storage == "bf16" else 1e-5, batch=args.batch, acc=int(args.acc),
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
        self.storage = lra.LRA_F32 if args.storage == "f32" else lra.LRA_BF16
        self.esize = 4 if args.storage == "f32" else 2
        self.Xt, _ = L.planted_torch(wl.d, wl.n, wl.sigma(), wl.seed, device=device)
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
        import torch
        X = self.Xt if self.Xt is not None else self.Xh.to(U.device)
        Xd = X.double()
        P = Xd @ U.double().T
        e = float((Xd * Xd).sum()) - float((P * P).sum())
        del Xd, P
        torch.cuda.empty_cache()
        return e

    def pass_bytes(self, kind, pav):
        return self.x_bytes + (self.wl.d + self.wl.n) * pav * 4

    def oracle_input(self):
        return self.to_host().numpy()


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

    def pass_bytes(self, kind, pav):
        wl = self.wl
        # compressed index + value of every non-zero, the line pointers, the
        # dense operand and the result (gathers of the operand hit L2)
        if kind == "xtw":
            return self.nnz * 8 + (wl.n + 1) * 8 + (wl.d + wl.n) * pav * 4
        return self.nnz * 8 + (wl.d + 1) * 8 + (wl.n + wl.d) * pav * 4

    def oracle_input(self):
        return self.xt()


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
            t_fixed, t_outer, lam, E = oracle_sample(wl, Xh, args, lam1, args.cpu_sample_outer, threads)
            Lstar = predicted_outer(wl, lam, E, args.eps)
            v = t_fixed + t_outer * Lstar
            sample_desc = (f"FP64 oracle on the same X and seeds: lambda_1 estimate + "
                           f"{args.cpu_sample_outer} outer iterations, extrapolated to {Lstar} outer "
                           f"iterations (sampled Ritz error, theory rate)")
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": "time-to-eps", "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "d": wl.d, "n": wl.n, "k": wl.k, "p": wl.p,
                   "storage": "csr" if wl.storage == "csr" else args.storage, "shift": args.shift,
                   "eps": args.eps},
        "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


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

    ctx = lra.lra_init(local)
    mat = src.create(ctx)
    stream = torch.cuda.ExternalStream(lra.lra_ctx_stream(ctx), device=device)
    U = torch.zeros(wl.k, wl.d, dtype=torch.float32, device=device)
    ritz = torch.zeros(wl.k, dtype=torch.float64, device=device)

    def one(rep):
        return lra.lra_solve(mat, wl.k, wl.p, args.eps, args.seed, opt, U, ritz, rep)

    for _ in range(args.warmup):
        one(lra.LraReport())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    reps = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rep = lra.LraReport()
        st = one(rep)
        reps.append((st, rep))
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    ms_step = ms_total / args.steps
    if world > 1:
        ms_step = max_over_ranks(ms_step, device)

    # accuracy of the last solve, off the clock (FP64 error against the
    # closed-form or stored reference optimum)
    ratio = src.err(U) / opt_val

    # roofline of the dominant kernel from its live CUDA-event timing
    peaks, peak_kind = measured_peaks()
    last = reps[-1][1]
    tot = {"xtw": sum(r.xtw_ms for _, r in reps), "xy": sum(r.xy_ms for _, r in reps),
           "inner": sum(r.inner_ms for _, r in reps)}
    cnt = {"xtw": sum(r.xtw_launches for _, r in reps), "xy": sum(r.xy_launches for _, r in reps),
           "inner": sum(r.inner_launches for _, r in reps)}
    cols = {"xtw": sum(r.xtw_cols for _, r in reps), "xy": sum(r.xy_cols for _, r in reps)}
    dom = max(tot, key=lambda k: tot[k])
    roof = None
    if dom in ("xtw", "xy") and cnt[dom] > 0:
        pav = cols[dom] / cnt[dom]
        bytes_l = src.pass_bytes(dom, pav)
        t_l = tot[dom] / cnt[dom] / 1e3
        hbm = peaks["hbm_gbs"] * 1e9
        if src.tensor:
            # dense X passes run on tensor cores: BF16 X with 2 BF16 MMAs per
            # k-step (hi/lo small operand), FP32 X as a BF16 pair with 3; the
            # executed tensor flops are compared with the measured sustained BF16 peak
            flops_l = 2.0 * wl.d * wl.n * pav
            mmas = 2 if args.storage == "bf16" else 3
            tens = peaks["bf16_tflops_sustained"] * 1e12 / mmas
            compute_bound = bytes_l / hbm < flops_l / tens
        else:
            compute_bound = False
        if compute_bound:
            roof = {"bound": "tensor", "achieved": flops_l / t_l / 1e12, "peak": tens / 1e12,
                    "unit": "TFLOP/s", "frac": flops_l / t_l / tens, "traffic": None}
        else:
            roof = {"bound": "hbm", "achieved": bytes_l / t_l / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": bytes_l / t_l / hbm, "traffic": None}
        names = {("xtw", True): "xtw_tc_kernel", ("xy", True): "xy_tc_kernel",
                 ("xtw", False): "spmm_xt_kernel", ("xy", False): "spmm_x_kernel"}
        roof["traffic"] = recorded_traffic(args.workload, names[(dom, src.tensor)])
        roof.update({"kernel": names[(dom, src.tensor)],
                     "launches": cnt[dom], "ms_per_launch": t_l * 1e3,
                     "algorithmic_bytes_per_launch": bytes_l,
                     "x_pass_gbs": bytes_l / t_l / 1e9, "peak_source": peak_kind})
    elif cnt["inner"] > 0:
        roof = {"bound": "latency", "achieved": None, "peak": None, "unit": "steps/s",
                "frac": None, "traffic": None,
                "kernel": "inner_csc_kernel" if wl.storage == "csr" else "svrg_inner_kernel"}

    # every timed kernel class: launches, time, X-pass GB/s (algorithmic bytes)
    per_kernel = {}
    for kk in ("xtw", "xy", "inner"):
        if cnt[kk] > 0:
            e = {"launches": cnt[kk], "ms_total": tot[kk], "ms_per_launch": tot[kk] / cnt[kk]}
            if kk in cols:
                pav = cols[kk] / cnt[kk]
                e["x_pass_gbs"] = src.pass_bytes(kk, pav) / (tot[kk] / cnt[kk] / 1e3) / 1e9
            if kk == "inner":
                steps = sum(r.inner_steps for _, r in reps)
                if steps > 0:
                    e["steps"] = steps
                    e["ns_per_step"] = tot[kk] * 1e6 / steps
                    # every CTA of the one-sample loop owns a column group on its
                    # own SM and takes all m steps: steps/s per SM = 1 / step time
                    e["steps_per_s_per_sm"] = 1e9 / e["ns_per_step"]
            per_kernel[kk] = e

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Uh = torch.empty(wl.k, wl.d, dtype=torch.float32, pin_memory=True)
        rh = torch.empty(wl.k, dtype=torch.float64, pin_memory=True)
        lra.lra_mat_destroy(mat)
        mat = None
        src.drop_device()
        torch.cuda.empty_cache()
        times = []
        for _ in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = src.create_from_host(ctx)
            lra.lra_solve(m2, wl.k, wl.p, args.eps, args.seed, opt, Uh, rh, lra.LraReport())
            lra.lra_mat_destroy(m2)
            times.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(times[1:]), "unit": "s",
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
        t_fixed, t_outer, lam, E = oracle_sample(wl, src.oracle_input(), args, None, args.cpu_sample_outer,
                                                 threads)
        Lg = last.outer_iters
        cpu = {"value": t_fixed + t_outer * Lg, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": (f"FP64 oracle on the same X and seeds: lambda_1 estimate ({t_fixed:.1f} s) "
                          f"+ {args.cpu_sample_outer} outer iterations ({t_outer:.2f} s each), "
                          f"extrapolated to the GPU run's {Lg} outer iterations")}

    if mat is not None:
        lra.lra_mat_destroy(mat)
    lra.lra_finalize(ctx)
    if rank == 0:
        line = {
            "metric": "time-to-eps", "value": ms_step / 1e3, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if storage_name == "csr" else args.storage, "data": "synthetic",
            "config": {"workload": args.workload, "d": wl.d, "n": wl.n, "k": wl.k, "p": wl.p,
                       "storage": storage_name, "shift": args.shift, "eps": args.eps, "batch": args.batch,
                       "acc": bool(args.acc), "partition": bool(args.partition),
                       "l2": "inputs larger than L2 (X %.2f GB per pass)" % (src.x_bytes / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy": {"ratio_err_over_opt": ratio, "outer_iters": last.outer_iters,
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
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Request-loop benchmark: a Poisson stream of rank-k requests of uneven
    d, n, k and storage type served by lra_submit / lra_poll, against the same
    stream run one job at a time with FP32 storage through lra_solve."""
    import threading

    import torch
    import paper_1607_02925_gb300 as lra

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
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

    # ---- served: continuous batching
    ctx = lra.lra_init(local)
    t0 = time.perf_counter()
    done_t = [None] * nreq
    results = [None] * nreq
    outstanding = {}
    lock = threading.Lock()

    def submitter():
        for j, q in enumerate(reqs):
            wait = t0 + arrivals[j] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            m = make(ctx, q, lra.LRA_BF16 if q["bf16"] else lra.LRA_F32)
            jid = lra.lra_submit(ctx, m, q["k"], 2 * q["k"], args.eps, 1000 + j, opt)
            with lock:
                outstanding[jid] = (j, m)

    th = threading.Thread(target=submitter)
    th.start()
    finished = 0
    while finished < nreq:
        with lock:
            items = list(outstanding.items())
        progressed = False
        for jid, (j, m) in items:
            q = reqs[j]
            U = torch.empty(q["k"], q["d"], device=dev)
            r = torch.empty(q["k"], dtype=torch.float64, device=dev)
            st = lra.lra_poll(ctx, jid, 0, U, r, allow=(4, 7, 8))
            if st in (7, 8):
                continue
            done_t[j] = time.perf_counter() - t0
            results[j] = (st, U.cpu().numpy(), r.cpu().numpy())
            with lock:
                del outstanding[jid]
            lra.lra_mat_destroy(m)
            finished += 1
            progressed = True
        if not progressed:
            time.sleep(0.0005)
    th.join()
    lat = np.array(done_t) - arrivals
    span = max(done_t) - arrivals[0]
    # sampled results re-run alone must be bitwise equal
    nchk = min(50, nreq)
    check = list(range(0, nreq, max(1, nreq // nchk)))[:nchk]
    equal = 0
    for j in check:
        q = reqs[j]
        m = make(ctx, q, lra.LRA_BF16 if q["bf16"] else lra.LRA_F32)
        U = torch.empty(q["k"], q["d"], device=dev)
        r = torch.empty(q["k"], dtype=torch.float64, device=dev)
        lra.lra_solve(m, q["k"], 2 * q["k"], args.eps, 1000 + j, opt, U, r)
        lra.lra_mat_destroy(m)
        equal += int(np.array_equal(U.cpu().numpy(), results[j][1]) and np.array_equal(r.cpu().numpy(), results[j][2]))
    lra.lra_finalize(ctx)

    # ---- baseline: one job at a time, FP32 storage, same arrival times
    ctx = lra.lra_init(local)
    tb = 0.0
    blat = []
    for j, q in enumerate(reqs):
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
    blat = np.array(blat)
    line = {
        "metric": "serve_latency", "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "requests": nreq, "mean_interarrival_ms": args.serve_mean_ms,
        "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
        "jobs_per_s": nreq / span, "bitwise_equal_alone": f"{equal}/{len(check)}",
        "statuses": sorted({int(r[0]) for r in results}),
        "baseline_one_at_a_time_f32": {"p50": float(np.percentile(blat, 50)),
                                        "p99": float(np.percentile(blat, 99)),
                                        "jobs_per_s": nreq / (tb - arrivals[0])},
        "config": {"workload": "planted small-gap spectrum rescaled to k; d in {256,1024,4096}, "
                               "n in {8192,65536,262144}, k in {5,10,20,50}, p = 2k, FP32/BF16 1:1",
                   "shift": "far", "eps": args.eps, "slots": int(os.environ.get("LRA_SERVE_SLOTS", "8"))},
        "data": "synthetic",
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.serve:
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_lra(args)


if __name__ == "__main__":
    sys.exit(main())
