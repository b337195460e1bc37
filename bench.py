#!/usr/bin/env python
"""bench.py -- posv TFLOP/s and time-to-solution at backward error <= 1e-13:
mixed precision + FP64 refinement vs plain FP64, on one GB300.

One step = one posv call (factor + solves + refinement) on the workload's
synthetic matrix, resident in HBM.  The default workload is the largest
single-GPU configuration: n = 65536, nrhs = 32, A = M M^T/n + 1e-2 I with FP8
e4m3 trailing updates (per-tile power-of-two scales) and FP64 refinement,
against the plain FP64 path on the same system.  A (34 GB) is far larger than
the 129 MB L2, so no flush is needed between steps.  TFLOP/s uses the nominal
count n^3/3 + 2 n^2 nrhs.  Every returned X is certified on the host by the
CPU oracle's Dot2 backward error.  Prints ONE JSON line; `extra_configs` holds
one timed solve of each other configuration (n = 1024; n = 32768 at
kappa = 1e2 .. 1e8 with BF16 and FP16 words; the autograd workload at
n = 8192; the paper's diag(1..N)).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c4|c2|...]
                  [--extra c1,c3,c5,c6|none]
  python bench.py --impl reference ...   (the CPU oracle, timed on host cores)

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the factorisation does not shard into independent units); value = all ranks'
flops / max-over-ranks time.
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

METRIC = ("posv TFLOP/s & time-to-solution at backward err ≤1e-13: mixed+IR vs FP64, "
          "1×GB300")

# workload -> (n, nrhs, matrix kind, kappa or shift, precision, words)
WORKLOADS = {
    "c1": dict(n=1024, nrhs=1, kind="gram", param=1.0, prec="fp32", words=1,
               desc="posv n=1024 nrhs=1, A = M M^T/n + I (one-kernel FP32-factor path)"),
    "c2": dict(n=16384, nrhs=64, kind="qlam", param=1e6, prec="fp16", words=2,
               desc="posv n=16384 nrhs=64, A = Q diag(logspace[1,1e6]) Q^T, B = A X_true"),
    "c3": dict(n=32768, nrhs=16, kind="qlam", param=1e4, prec="fp16", words=2,
               desc="posv n=32768 nrhs=16, A = Q diag(logspace[1,kappa]) Q^T"),
    "c4": dict(n=65536, nrhs=32, kind="gram32", param=1e-2, prec="fp8", words=1,
               desc="posv n=65536 nrhs=32, A = M M^T/n + 1e-2 I (product formed in FP32), "
                    "FP8 e4m3 trailing updates with per-128x128-tile power-of-two scales"),
    "c5": dict(n=8192, nrhs=16, kind="gram", param=1.0, prec="bf16", words=2,
               desc="autograd forward+backward n=8192 nrhs=16, A = M M^T/n + I, B ~ N(0,1), "
                    "loss 0.5||X||^2", rhs="normal"),
    "c6": dict(n=16384, nrhs=1, kind="diag", param=0.0, prec="bf16", words=1,
               desc="posv n=16384 nrhs=1, the paper's A = diag(1..N), b = ones (x_i = 1/i)"),
}

# The n = 32768 condition-number ladder: for each kappa, the split words of the
# BF16 and of the FP16 tensor-core factor (more words as kappa grows).
C3_LADDER = [(1e2, {"bf16": 1, "fp16": 1}), (1e4, {"bf16": 2, "fp16": 2}),
             (1e6, {"bf16": 3, "fp16": 2}), (1e8, {"bf16": 3, "fp16": 2})]

FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def nominal_flops(n, nrhs):
    return n ** 3 / 3.0 + 2.0 * n * n * nrhs


def max_over_ranks(values, world, device="cpu"):
    """Elementwise max of a list of floats over all ranks (replicas run the same
    steps; the slowest rank sets the job time)."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replica_value(world, flops_per_step, steps, t_max_s):
    """Whole-job TFLOP/s of `world` independent replicas, each doing `steps`
    steps of `flops_per_step`, in the max-over-ranks time t_max_s."""
    return world * flops_per_step * steps / t_max_s / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def log(msg):
    print("[bench %s] %s" % (time.strftime("%H:%M:%S"), msg), file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                # a throttle reason counts even where a number is unreadable;
                # the numbers of a sample count only if all three are readable
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
                try:
                    vals = float(p[1]), float(p[2]), float(p[3])
                except ValueError:
                    continue
                sm.append(vals[0])
                smax.append(vals[1])
                power.append(vals[2])
            os.unlink(self.path)
        except Exception:
            pass
        busy = [v for v in sm if v > 0] or [0.0]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- inputs
def make_inputs(w, device, seed=0, Q=None):
    """(A, X_true or None, B) on `device`; A symmetric (row- and column-major
    forms coincide).  Q: an orthogonal factor to reuse for the Q-lambda kind."""
    import torch

    from paper_2601_14466_gb300 import inputs

    n, nrhs = w["n"], w["nrhs"]
    if w["kind"] == "diag":  # the paper's matrix: A = diag(1..N), b = ones, x_i = 1/i
        A, B = inputs.diag_workload(n, device=device)
        Xt = (1.0 / torch.arange(1, n + 1, dtype=torch.float64, device=device)).reshape(n, 1)
        torch.cuda.synchronize()
        return A, Xt, B
    if w["kind"] == "qlam":
        A = inputs.from_q(Q, w["param"]) if Q is not None else \
            inputs.q_lambda(n, w["param"], seed=seed, device=device)
    else:
        A = inputs.gram_shift(n, w["param"], seed=seed, device=device,
                              fp32_product=(w["kind"] == "gram32"))
    if w.get("rhs") == "normal":
        B = inputs.normal(n, nrhs, seed=seed + 1, device=device)  # column-major
        torch.cuda.synchronize()
        return A, None, B
    Xt = inputs.uniform(n, nrhs, seed=seed + 1, device=device)
    B = inputs.rhs_from(A, Xt)
    torch.cuda.synchronize()
    return A, Xt, B


def kappa_of_gram(A, shift, iters=20, seed=7):
    """kappa of A = M M^T/n + shift*I, as far as it can be measured at this
    size: lambda_max by power iteration (FP64 products, a lower bound that the
    iteration approaches from below) and lambda_min >= shift (M M^T/n is
    positive semidefinite; for square M its smallest eigenvalue is O(1/n^2),
    so lambda_min is the shift up to that and the FP32 rounding of the
    product).  A diagnostic outside the timed region."""
    import torch

    g = torch.Generator(device=A.device).manual_seed(seed)
    v = torch.randn(A.shape[0], dtype=torch.float64, device=A.device, generator=g)
    v /= v.norm()
    lam = 0.0
    for _ in range(iters):
        w = A @ v
        lam = float(torch.dot(v, w).item())
        v = w / w.norm()
    return {"lambda_max_power_iteration": lam, "power_iterations": iters,
            "lambda_min_lower_bound": shift, "kappa": lam / shift,
            "method": "lambda_max by power iteration (FP64 products); lambda_min = the "
                      "shift up to O(1/n^2), since M M^T/n is positive semidefinite"}


def host_f(t):
    """A device (n x m) tensor as a column-major float64 NumPy array."""
    import numpy as np

    return np.asfortranarray(t.detach().double().cpu().numpy())


def certify(A_host, X, B):
    """The CPU oracle's normwise backward error of X (Dot2 residual), max over
    the columns; A_host: the symmetric matrix as a NumPy array (either order)."""
    import oracle

    Af = A_host if A_host.flags.f_contiguous else A_host.T  # symmetric: same matrix
    eta, _ = oracle.bwd_err_rows(Af, host_f(X), host_f(B))
    return eta


# ----------------------------------------------------------------------------- CPU oracle leg
def _oracle_sample_inputs(w, n_s):
    import numpy as np

    from paper_2601_14466_gb300 import inputs

    nrhs = w["nrhs"]
    if w["kind"] == "diag":
        A, B = (np.asfortranarray(t.numpy()) for t in inputs.diag_workload(n_s))
        return A, B
    if w["kind"] == "qlam":
        A = inputs.q_lambda(n_s, w["param"], seed=11).numpy()
    else:
        A = inputs.gram_shift(n_s, w["param"], seed=11).numpy()  # same construction, FP64
    X = inputs.uniform(n_s, nrhs, seed=12).numpy()
    return A, np.asfortranarray(A @ X)


def oracle_sample_n(w):
    # one solve of the sample takes about a second on 16 Grace cores
    return min(w["n"], 4096)


def cpu_oracle_timed(w, steps, warmup):
    """Time the oracle (as it stands) on `warmup` + `steps` solves of a bounded
    sample of the workload: the same construction at a reduced n, nrhs
    unchanged.  Returns the per-solve times of the timed solves."""
    import oracle

    n_s = oracle_sample_n(w)
    A, B = _oracle_sample_inputs(w, n_s)
    oracle.build()
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        _, info = oracle.posv(A, B)
        dt = time.perf_counter() - t0
        if info != 0:
            raise RuntimeError("oracle posv failed on the sample (info=%d)" % info)
        if k >= warmup:
            times.append(dt)
    return n_s, times


def cpu_baseline(w, steps=2):
    import oracle

    n_s, times = cpu_oracle_timed(w, steps, 0)
    t = statistics.mean(times)
    F = nominal_flops(n_s, w["nrhs"])
    return {"value": F / t / 1e12, "unit": "TFLOP/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "oracle posv at n=%d nrhs=%d (same construction, %d timed solves, "
                      "%.3f s each); at the workload's n=%d the same rate would take %.0f s "
                      "per solve (n^3 extrapolation, not run)"
                      % (n_s, w["nrhs"], len(times), t, w["n"],
                         t * nominal_flops(w["n"], w["nrhs"]) / F)}


# ----------------------------------------------------------------------------- GPU helpers
def _device():
    import torch

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    return dev


def _eta(jmg, Acm, X, B, anorm):
    _, cm = jmg.residual(Acm, X, B)
    cm = cm.cpu()
    return float((cm[0] / (anorm * cm[1] + cm[2])).max())


def _cw_bwd_err(jmg, torch, A, Acm, X, B):
    """Componentwise (Oettli-Prager) backward error of the returned X,
    max_ij |r_ij| / (|A| |x_j| + |b_j|)_i, with R from the exact split product
    (one rounding per element) and the denominator from FP64 absolute values;
    a diagnostic beside the normwise figure, taken at n <= 16384 only."""
    if A.shape[0] > 16384:
        return None
    try:
        R, _, err = jmg.residual_split(Acm, X, B)
        D = torch.abs(A) @ torch.abs(X) + torch.abs(B)
        Ra = torch.abs(R)
        q = torch.where(D > 0, Ra / torch.where(D > 0, D, torch.ones_like(D)),
                        torch.where(Ra > 0, torch.full_like(Ra, float("inf")), torch.zeros_like(Ra)))
        if int(err.item()) != 0:
            return None
        return float(q.max().item())
    except Exception:  # a diagnostic: never costs the measurement its line
        return None


def _timed(stream, fn):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def _fp64_posv(jmg, A, B, stream, steps, warmup=0, nb=128):
    """Plain FP64 posv on a scratch copy of A (restored before every step,
    outside the timed region); returns (ms per timed step, X)."""
    import torch

    Awork = torch.empty_like(A)
    ms, X = [], None
    for k in range(warmup + steps):
        Awork.copy_(A)
        dt, (X, _) = _timed(stream, lambda: jmg.posv(Awork.t(), B, prec="fp64", overwrite_a=True,
                                                     check=False, nb=nb))
        if k >= warmup:
            ms.append(dt)
    del Awork
    return ms, X


def _roofline_objects(n, nrhs, prec, words, infos, steps_ms, peaks, resid_mode):
    """Per-launch rooflines of the solve and the residual product, from the
    library's CUDA events inside the timed steps, and the factorisation's
    tensor-core rate.  Returns (dominant, others)."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    src = "of measured (MEASURED_PEAKS.json)" if peaks else "of fallback"
    n_sol = sum(si.n_solve for si in infos)
    t_sol = sum(si.t_solve_gpu_ms for si in infos)
    n_res = sum(si.n_resid for si in infos)
    t_res = sum(si.t_resid_gpu_ms for si in infos)
    t_fac = sum(si.t_factor_gpu_ms for si in infos)
    total_ms = steps_ms * len(infos)
    objs = {}
    if n_sol:
        # one triangular solve with the FP32 factor: the lower triangle of L read
        # once, the n x nrhs block read and written once
        sol_bytes = n * (n + 1) / 2 * 4 + 2 * n * nrhs * 4
        launch_ms = t_sol / (2 * n_sol)
        ach = sol_bytes / (launch_ms / 1e3) / 1e9
        objs["solve"] = {"kernel": "triangular solve with the FP32 factor (one launch per "
                                   "direction)",
                         "bound": "hbm", "achieved": round(ach, 2), "peak": hbm, "unit": "GB/s",
                         "frac": round(ach / hbm, 4), "peak_source": src,
                         "algorithmic_bytes_per_launch": sol_bytes,
                         "launch_ms": round(launch_ms, 4), "launches": 2 * n_sol,
                         "share_of_step": round(t_sol / total_ms, 4)}
    if n_res:
        launch_ms = t_res / n_res
        if resid_mode != "fp64":
            # split product: 36 slice pairs of BF16 MMA work; the slices of A
            # (8 x 2 bytes per element of the full matrix) are streamed once
            mma = 36 * 2.0 * n * n * nrhs
            sl_bytes = 16.0 * n * n
            t_mma = mma / (bf16 * 1e12)
            t_hbm = sl_bytes / (hbm * 1e9)
            if t_hbm >= t_mma:
                ach = sl_bytes / (launch_ms / 1e3) / 1e9
                o = {"bound": "hbm", "achieved": round(ach, 2), "peak": hbm, "unit": "GB/s",
                     "algorithmic_bytes_per_launch": sl_bytes}
            else:
                ach = mma / (launch_ms / 1e3) / 1e12
                o = {"bound": "tensor", "achieved": round(ach, 2), "peak": bf16,
                     "unit": "TFLOP/s", "algorithmic_flops_per_launch": mma}
            o["kernel"] = "split FP64-accurate product A X (BF16 tensor cores, exact windows)"
            o["fp64_equivalent_tflops"] = round(2.0 * n * n * nrhs / (launch_ms / 1e3) / 1e12, 3)
        else:
            ach = 2.0 * n * n * nrhs / (launch_ms / 1e3) / 1e12
            o = {"kernel": "FP64 product A X (CUDA cores)", "bound": "alu", "achieved": round(ach, 3),
                 "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s"}
        o.update({"frac": round(o["achieved"] / o["peak"], 4), "peak_source": src,
                  "launch_ms": round(launch_ms, 4), "launches": n_res,
                  "share_of_step": round(t_res / total_ms, 4)})
        objs["residual_product"] = o
    if t_fac > 0:
        pairs = {1: 1, 2: 3, 3: 6}.get(words, 1) if prec != "fp8" else 1
        mma_f = pairs * n ** 3 / 3.0
        pk = bf16 * (2.0 if prec == "fp8" else 1.0)  # e4m3: twice the 16-bit rate (nominal ratio)
        fac_ms = t_fac / len(infos)
        objs["factor"] = {"kernels": "diagonal blocks, panel solves, word split / FP8 quantise, "
                                     "tensor-core trailing updates",
                          "bound": "tensor", "unit": "TFLOP/s",
                          "achieved": round(mma_f * sum(si.factor_tries for si in infos) /
                                            len(infos) / (fac_ms / 1e3) / 1e12, 3),
                          "peak": pk, "peak_source": src, "ms": round(fac_ms, 3),
                          "share_of_step": round(t_fac / total_ms, 4),
                          "note": "tensor-core MMA flops of the trailing updates (%d word pairs, "
                                  "every factorisation of the step) over the factorisation time"
                                  % pairs}
        objs["factor"]["frac"] = round(objs["factor"]["achieved"] / pk, 4)
    per_launch = {k: v for k, v in objs.items() if k != "factor"}
    dom = max(per_launch, key=lambda k: per_launch[k]["share_of_step"]) if per_launch else None
    return dom, objs


# ----------------------------------------------------------------------------- main GPU arm
def run_main(args, w, rank, world):
    import numpy as np
    import torch

    from paper_2601_14466_gb300 import jmg

    dev = _device()
    jmg.load()
    n, nrhs = w["n"], w["nrhs"]
    prec, words = args.prec or w["prec"], args.words or w["words"]
    t0 = time.time()
    A, Xt, B = make_inputs(w, dev)
    log("inputs n=%d ready in %.1f s" % (n, time.time() - t0))
    Acm = A.t()  # symmetric: the transpose view is the column-major matrix
    kw = dict(prec=prec, words=words, nb=args.nb, maxit=args.maxit, refine=args.refine,
              resid=args.resid)
    opts = jmg.default_options(prec=prec, words=words, nb=args.nb,
                               resid={"auto": 0, "fp64": 1, "split": 2}[args.resid])
    work = jmg.workspace(jmg.OP_POSV, n, nrhs, opts, dev)
    stream = torch.cuda.current_stream(dev)
    F = nominal_flops(n, nrhs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- mixed precision + FP64 refinement
    for _ in range(args.warmup):
        X, si = jmg.posv(Acm, B, work=work, **kw)
    barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    l0 = jmg.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    infos = []
    ev[0].record(stream)
    for k in range(args.steps):
        X, si = jmg.posv(Acm, B, work=work, timing=True, **kw)
        ev[k + 1].record(stream)
        infos.append(si)
    barrier()
    launches = jmg.launch_count() - l0
    clocks = sampler.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_mixed = sum(step_ms) / 1e3
    log("mixed: %.1f ms/step" % (t_mixed * 1e3 / args.steps))
    anorm = float(jmg.norm_inf(Acm).item())
    eta = _eta(jmg, Acm, X, B, anorm)
    eta_cw = _cw_bwd_err(jmg, torch, A, Acm, X, B)
    fwd = float(((X - Xt).abs().max() / Xt.abs().max()).item()) if Xt is not None else None

    # ---- host copy of A: certification by the oracle, and the end-to-end leg
    # (before the FP64 leg, whose minutes of FP64 work would heat the GPU
    # under the end-to-end timing)
    A_h = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    A_h.copy_(A)
    X_keep, B_keep = X.clone(), B.clone()

    # ---- end to end through the public API with host buffers: jmg_posv_host
    # copies A and B from page-locked host memory, solves, and copies X back,
    # all inside the timed region
    e2e_steps = args.e2e_steps
    t_e2e, e2e_bytes, e2e_clocks = None, (0, 0), None
    if e2e_steps > 0:
        B_h = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).t()
        B_h.copy_(B)
        X_h = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).t()
        del work  # the host call stages A and B in front of its own posv workspace
        torch.cuda.empty_cache()
        work_h = jmg.workspace(jmg.OP_POSV_HOST, n, nrhs, opts, dev)
        e2e_ms = []
        e2e_sampler = ClockSampler(dev.index)
        for k in range(1 + e2e_steps):
            if k == 1:
                e2e_sampler.start()
            dt, (_, sh) = _timed(stream, lambda: jmg.posv_host(A_h.t(), B_h, out=X_h, work=work_h,
                                                               **kw))
            if k > 0:
                e2e_ms.append(dt)
                e2e_bytes = (sh.h2d_bytes, sh.d2h_bytes)
        e2e_clocks = e2e_sampler.stop()
        t_e2e = sum(e2e_ms) / 1e3
        del work_h
        torch.cuda.empty_cache()
        log("e2e: %.1f ms/step" % (t_e2e * 1e3 / e2e_steps))

    # ---- plain FP64 GPU path on the same system
    f64_steps = args.fp64_steps
    t_f64, X64 = None, None
    if f64_steps > 0:
        f64_ms, X64 = _fp64_posv(jmg, A, B, stream, f64_steps, nb=args.nb)
        t_f64 = sum(f64_ms) / 1e3
        log("fp64: %.1f ms/step" % (t_f64 * 1e3 / f64_steps))

    # ---- across ranks: max time
    t_mixed, tf, te = max_over_ranks([t_mixed, t_f64 or 0.0, t_e2e or 0.0], world, dev)
    t_f64 = tf if f64_steps > 0 else None
    t_e2e = te if e2e_steps > 0 else None

    # ---- certification of the returned X by the CPU oracle (Dot2 residual)
    t0 = time.time()
    A_np = A_h.numpy()
    eta_or = certify(A_np, X_keep, B_keep) if rank == 0 else None
    eta64_or = certify(A_np, X64, B_keep) if (rank == 0 and X64 is not None) else None
    log("oracle certification: %.1f s" % (time.time() - t0))
    kappa = kappa_of_gram(Acm, w["param"]) if w["kind"] in ("gram", "gram32") else (
        {"kappa": w["param"], "method": "by construction (log-spaced spectrum)"}
        if w["kind"] == "qlam" else None)

    value = replica_value(world, F, args.steps, t_mixed)
    peaks = load_peaks()
    steps_ms = t_mixed * 1e3 / args.steps
    dom, objs = _roofline_objects(n, nrhs, prec, words, infos, steps_ms, peaks, args.resid)
    roof = dict(objs[dom]) if dom else None
    if roof is not None:
        roof["traffic"] = traffic_per_launch(dom, n, nrhs)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_mixed * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (%s%s tensor-core factor)" % (prec, "x%d" % words if prec != "fp8" else ""),
        "data": "synthetic, seeded (torch.Generator); A resident in HBM, larger than L2",
        "config": {"workload": w["desc"], "n": n, "nrhs": nrhs, "prec": prec, "words": words,
                   "nb": args.nb, "tol": 1e-13, "refine": args.refine,
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (A = %.2f GB), no flush" % (n * n * 8 / 1e9)},
        "time_to_solution_ms": round(t_mixed * 1e3 / args.steps, 3),
        "bwd_err_oracle": eta_or, "bwd_err": eta, "bwd_err_componentwise": eta_cw,
        "fwd_err": fwd, "kappa": kappa,
        "iters": [si.iters for si in infos],
        "refine_used": ["ir", "pcg", "auto"][infos[-1].refine_used] if infos[-1].refine_used >= 0 else None,
        "shift": infos[-1].shift, "factor_tries": infos[-1].factor_tries,
        "eta_hist": [float("%.3e" % e) for e in infos[-1].eta_hist],
        "phases_ms": {"factor_gpu": round(statistics.mean(si.t_factor_gpu_ms for si in infos), 3),
                      "solves_gpu": round(statistics.mean(si.t_solve_gpu_ms for si in infos), 3),
                      "residual_products_gpu": round(statistics.mean(si.t_resid_gpu_ms for si in infos), 3)},
        "roofline": roof,
        "kernels": {k: v for k, v in objs.items() if k != dom},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "clocks": clocks,
    }
    if t_f64 is not None:
        fp64_value = replica_value(world, F, f64_steps, t_f64)
        out["fp64"] = {"value": round(fp64_value, 4), "unit": "TFLOP/s",
                       "ms_per_step": round(t_f64 * 1e3 / f64_steps, 3), "steps": f64_steps,
                       "bwd_err_oracle": eta64_or,
                       "frac_of_fp64_nominal": round(fp64_value / world / FP64_NOMINAL_TFLOPS, 4)}
        out["speedup_mixed_vs_fp64"] = round((t_f64 / f64_steps) / (t_mixed / args.steps), 3)
    if t_e2e is not None:
        out["e2e"] = {"value": round(replica_value(world, F, e2e_steps, t_e2e), 4), "unit": "TFLOP/s",
                      "ms_per_step": round(t_e2e * 1e3 / e2e_steps, 3),
                      "h2d_bytes_per_step": e2e_bytes[0], "d2h_bytes_per_step": e2e_bytes[1],
                      "call": "jmg_posv_host (A and B host->device, X device->host, "
                              "page-locked host buffers)", "clocks": e2e_clocks}
    del A, A_h, B, X, X_keep, B_keep, X64
    torch.cuda.empty_cache()
    return out


# DRAM traffic (read + write) per launch of the dominant kernel, from one ncu
# capture, as a multiple of the algorithmic bytes at the captured size; the
# kernel reads each byte of L once, so its traffic scales with the algorithmic
# bytes.  None where the kernel changed since the capture.
# From the full captures of both kernels at n = 8192, nrhs = 32 (FP8 posv):
# residual product 1.0871 GB read+written for 1.0737 GB of slices, solve
# 141.2 MB for 136.3 MB.
TRAFFIC_RATIO = {"solve": 1.036, "residual_product": 1.012}


def traffic_per_launch(kind, n, nrhs):
    r = TRAFFIC_RATIO.get(kind)
    if r is None:
        return None
    if kind == "solve":
        return int(r * (n * (n + 1) / 2 * 4 + 2 * n * nrhs * 4))
    return int(r * 16.0 * n * n)


# ----------------------------------------------------------------------------- extra configs
def _one_config(jmg, torch, dev, stream, A, Xt, B, prec, words, steps=1, warmup=1, nb=128):
    """Timed mixed solve(s) of one configuration; returns a dict (ms, TFLOP/s,
    iterations, backward errors) and X."""
    n, nrhs = B.shape
    Acm = A.t()
    opts = jmg.default_options(prec=prec, words=words, nb=nb)
    work = jmg.workspace(jmg.OP_POSV, n, nrhs, opts, dev)
    ms, si, X = [], None, None
    for k in range(warmup + steps):
        dt, (X, si) = _timed(stream, lambda: jmg.posv(Acm, B, prec=prec, words=words, nb=nb,
                                                      work=work, check=False))
        if k >= warmup:
            ms.append(dt)
    del work
    t = statistics.mean(ms)
    d = {"prec": prec, "words": words if prec != "fp8" else None, "ms": round(t, 3),
         "tflops": round(nominal_flops(n, nrhs) / (t / 1e3) / 1e12, 3), "steps": steps,
         "status": si.status, "iters": si.iters,
         "refine_used": ["ir", "pcg", "auto"][si.refine_used] if si.refine_used >= 0 else None,
         "factor_tries": si.factor_tries, "bwd_err": si.bwd_err}
    if Xt is not None:
        d["fwd_err"] = float(((X - Xt).abs().max() / Xt.abs().max()).item())
    return d, X


def _c_abi_small_ms(jmg, torch, A, B, stream, steps=20, warmup=5):
    """The one-kernel path timed through the C ABI itself (jmg_posv with
    pre-made pointers, options and workspace), without the Python binding's
    per-call tensor set-up: the median of `steps` event-timed calls."""
    import ctypes

    n, nrhs = B.shape
    o = jmg.default_options(prec="fp32")
    work = jmg.workspace(jmg.OP_POSV, n, nrhs, o, A.device)
    lib = jmg.load()
    X = jmg.colmajor_copy(B)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = jmg.Stats()
    args = (n, nrhs, A.data_ptr(), n, X.data_ptr(), n, jmg.JMG_F64, info.data_ptr(),
            ctypes.byref(o), ctypes.byref(st), work.data_ptr(), work.numel(),
            ctypes.c_void_p(stream.cuda_stream))
    ms = []
    for k in range(warmup + steps):
        X.copy_(B)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = lib.jmg_posv(*args)
        e1.record(stream)
        e1.synchronize()
        if rc != 0:
            return None
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
    return round(statistics.median(ms), 4)


def run_extras(args, which):
    import numpy as np
    import torch

    from paper_2601_14466_gb300 import inputs, jmg

    dev = _device()
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name in which:
        t0 = time.time()
        if name in ("c1", "c6"):
            w = WORKLOADS[name]
            A, Xt, B = make_inputs(w, dev)
            A_np = host_f(A)
            small = w["n"] <= 2048
            d, X = _one_config(jmg, torch, dev, stream, A, Xt, B, w["prec"], w["words"],
                               steps=10 if small else 3, warmup=3 if small else 1)
            d["bwd_err_oracle"] = certify(A_np, X, B)
            if w["prec"] == "fp32":
                d["c_abi_ms"] = _c_abi_small_ms(jmg, torch, A, B, stream)
            if w["prec"] == "fp32":  # the tensor-core path on the same system, for context
                d2, X2 = _one_config(jmg, torch, dev, stream, A, Xt, B, "bf16", 1, steps=5,
                                     warmup=2)
                d2["bwd_err_oracle"] = certify(A_np, X2, B)
                d["tensor_core_path_bf16"] = d2
                del X2
            f64_ms, X64 = _fp64_posv(jmg, A, B, stream, 3, warmup=1)
            t64 = statistics.mean(f64_ms)
            out[name] = {"workload": w["desc"], "n": w["n"], "nrhs": w["nrhs"], "mixed": d,
                         "fp64": {"ms": round(t64, 3),
                                  "tflops": round(nominal_flops(w["n"], w["nrhs"]) / (t64 / 1e3) / 1e12, 3),
                                  "steps": 3, "bwd_err_oracle": certify(A_np, X64, B)},
                         "speedup_mixed_vs_fp64": round(t64 / d["ms"], 3)}
            if name == "c6":
                i = np.arange(1, w["n"] + 1, dtype=np.float64)
                out[name]["max_rel_err_vs_1_over_i"] = float(
                    np.max(np.abs(host_f(X)[:, 0] * i - 1.0)))
            del A, B, X, X64
        elif name == "c3":
            w = dict(WORKLOADS["c3"])
            Q = inputs.q_factor(w["n"], seed=0, device=dev)
            log("c3: Q ready in %.1f s" % (time.time() - t0))
            rows = []
            for kappa, words in C3_LADDER:
                w["param"] = kappa
                A, Xt, B = make_inputs(w, dev, Q=Q)
                A_np = host_f(A)
                row = {"kappa": kappa}
                for prec in ("bf16", "fp16"):
                    d, X = _one_config(jmg, torch, dev, stream, A, Xt, B, prec, words[prec])
                    d["bwd_err_oracle"] = certify(A_np, X, B)
                    row[prec] = d
                    del X
                f64_ms, X64 = _fp64_posv(jmg, A, B, stream, 1)
                row["fp64"] = {"ms": round(f64_ms[0], 3),
                               "tflops": round(nominal_flops(w["n"], w["nrhs"]) / (f64_ms[0] / 1e3) / 1e12, 3),
                               "steps": 1, "bwd_err_oracle": certify(A_np, X64, B)}
                for prec in ("bf16", "fp16"):
                    row[prec]["speedup_vs_fp64"] = round(f64_ms[0] / row[prec]["ms"], 3)
                rows.append(row)
                del A, B, Xt, X64, A_np
                torch.cuda.empty_cache()
                log("c3 kappa=%g done" % kappa)
            del Q
            out["c3"] = {"workload": "posv n=32768 nrhs=16, A = Q diag(logspace[1,kappa]) Q^T, "
                                     "one Q for every kappa", "n": w["n"], "nrhs": w["nrhs"],
                         "ladder": rows}
        elif name == "c5":
            out["c5"] = run_grad(args, WORKLOADS["c5"])
        torch.cuda.empty_cache()
        log("%s done in %.1f s" % (name, time.time() - t0))
    return out


def run_grad(args, w):
    """Forward + backward of the differentiable solve (autograd.SPDSolve) for
    loss = 0.5 ||X||_F^2: mixed forward (adjoint solve against the kept factor)
    vs the FP64 forward; the gradient checked by central differences of the FP64
    forward on 8 seeded entries and against the oracle's adjoint."""
    import numpy as np
    import torch

    import oracle
    from paper_2601_14466_gb300 import autograd, jmg

    dev = _device()
    n, nrhs = w["n"], w["nrhs"]
    prec, words = w["prec"], w["words"]
    A, _, B = make_inputs(w, dev)
    stream = torch.cuda.current_stream(dev)

    def step(p):
        Ad = A.clone().requires_grad_(True)
        Bd = B.clone().requires_grad_(True)

        def f():
            X = autograd.solve(Ad, Bd, p, words)
            (0.5 * (X * X).sum()).backward()
            return X

        dt, X = _timed(stream, f)
        return dt, Ad.grad, Bd.grad, X

    res = {}
    for p in (prec, "fp64"):
        step(p)
        res[p] = statistics.mean(step(p)[0] for _ in range(3))
    _, G, GB, X = step(prec)
    # the oracle's adjoint: Abar = -(Bbar X^T + X Bbar^T)/2, Bbar = A^{-1} X
    A_np = host_f(A)
    Xo, info = oracle.posv(A_np, host_f(B))
    _, Bbo, Abo, _ = oracle.grad(A_np, host_f(B), Xo)
    grad_err = float(np.abs(host_f(G) - Abo).max() / np.abs(Abo).max())
    rng = np.random.default_rng(33)
    h, worst = 1e-6, 0.0
    for _ in range(8):
        i, j = sorted(rng.integers(0, n, size=2))[::-1]
        E = torch.zeros_like(A)
        E[i, j] = h
        E[j, i] = h

        def loss(M):
            Xf, _ = jmg.posv(M.t(), B, prec="fp64")
            return 0.5 * float((Xf * Xf).sum().item())

        fd = (loss(A + E) - loss(A - E)) / (2 * h)
        want = float(G[i, j] + G[j, i]) if i != j else float(G[i, i])
        worst = max(worst, abs(fd - want) / max(1.0, abs(want)))
    F = nominal_flops(n, nrhs) + 2.0 * n * n * nrhs  # forward + adjoint solve
    return {"workload": w["desc"], "n": n, "nrhs": nrhs, "prec": prec, "words": words,
            "ms": round(res[prec], 3), "tflops": round(F / (res[prec] / 1e3) / 1e12, 3),
            "fp64_ms": round(res["fp64"], 3),
            "speedup_mixed_vs_fp64": round(res["fp64"] / res[prec], 3),
            "bwd_err_oracle": certify(A_np, X, B),
            "grad_max_rel_err_vs_oracle": grad_err,
            "fd_max_rel_err_8_entries": worst}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--extra", default="c1,c6,c5,c3",
                    help="comma-separated extra configurations (one timed solve each), or none")
    ap.add_argument("--prec", default=None)
    ap.add_argument("--words", type=int, default=None)
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--kappa", type=float, default=None)
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--refine", default="auto", choices=["ir", "pcg", "auto"])
    ap.add_argument("--resid", default="auto", choices=["auto", "fp64", "split"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.kappa is not None:
        w["param"] = args.kappa
        w["desc"] = w["desc"].replace("kappa", "%g" % args.kappa)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle

        # each step is one oracle solve of a bounded sample of the workload
        n_s, times = cpu_oracle_timed(w, args.steps, args.warmup)
        t = statistics.mean(times)
        value = nominal_flops(n_s, w["nrhs"]) / t / 1e12
        sample = ("oracle posv at n=%d nrhs=%d (same construction): %d warm-up and %d timed "
                  "solves, %.3f s each" % (n_s, w["nrhs"], args.warmup, len(times), t))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic, seeded",
            "config": {"workload": w["desc"] + " (bounded CPU sample: " + sample + ")",
                       "n": w["n"], "nrhs": w["nrhs"], "sample_n": n_s},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }))
        return 0

    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "c5":
        _device()
        out = run_grad(args, w)
        out.update({"metric": METRIC + " [differentiation workload: forward+backward]",
                    "value": out["tflops"], "unit": "TFLOP/s", "n_gpus": world,
                    "steps": 3, "warmup": 1, "ms_per_step": out["ms"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None})
    else:
        out = run_main(args, w, rank, world)
        extras = [e for e in args.extra.split(",") if e and e != "none" and e != args.workload]
        if extras and world == 1:
            out["extra_configs"] = run_extras(args, extras)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
