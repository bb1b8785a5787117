"""Benchmark: polynomial evaluations/s of the fast polynomial evaluator
(Algorithm A_p of arXiv 2211.06320) on the GPU, at d = 2^20.

Workload (default): d = 2^20, a_k uniform in the unit disk (seed 1), 2^20
sphere-uniform points per GPU, p = 53, FP64.  A step is one fpe_eval call over
all points (locate, bucket, window sums, valuation power); the polynomial is
preconditioned once before timing (reported separately, as the paper does).

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own
2^20 points of the same polynomial (weak scaling, no collective on the data
path); value = all ranks' evaluations / max-over-ranks time.

--impl reference times the CPU oracle (the plain restatement of the method)
on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "polynomial evaluations/s at d=2^20 (FPE vs GPU Horner, same accuracy), % of roofline"
TC_FLOPS_PER_SUBTILE = 2.0 * 128 * 64 * 880
UNIT = "evals/s"


# DRAM bytes per launch of the window-sum kernels from one ncu capture of this
# workload (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel sources it was taken on: the file records their SHA-256.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_unit_disk_d2pow20.txt")
KERNEL_SOURCES = ["fpe_eval.cu", "fpe_device.cuh", "fpe_internal.h", "fpe_window.cuh", "fpe_tc.cu",
                  "fpe_tc_arith.cuh", "fpe_tc05.cuh"]


def kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2211_06320_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel: str):
    """(bytes per launch, note) from the ncu record, or (None, why not)."""
    try:
        lines = [ln.split() for ln in open(TRAFFIC_FILE) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None, "no ncu traffic record"
    sha = kernel_sources_sha()
    for parts in lines:
        if len(parts) >= 3 and parts[0] == kernel:
            if parts[2] != sha:
                return None, "ncu traffic record predates the current kernel sources"
            return float(parts[1]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one full-size launch"
    return None, "no ncu traffic record for " + kernel


def measured_bf16_peak():
    """Dense bf16 TFLOP/s of the GB300s (measured cuBLAS burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops"])
        return v, "measured: MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 GEMM burst on this pool's GB300s)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback: 1.9 PFLOP/s bf16 burst (one earlier GB300 measurement)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fpe", choices=["fpe", "reference"])
    ap.add_argument("--points", type=int, default=1 << 20)
    ap.add_argument("--degree", type=int, default=1 << 20)
    ap.add_argument("--no-extras", action="store_true", help="skip Horner baselines, accuracy and CPU legs")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch parameters (no autotuning)")
    return ap.parse_args()


def workload(args, rank: int = 0, world: int = 1):
    """The polynomial and this rank's points.  Under torchrun the ranks share
    one point set of world x points points (the same coefficients, the
    points drawn after them from the same generator), split by
    lambda-sorted round-robin buckets (sharding.lambda_round_robin), so each
    rank gets about `points` points and a like share of the window work."""
    import workloads as W
    from paper_2211_06320_gb300.sharding import lambda_round_robin
    wl = W.unit_disk_d2pow20(n_points=args.points * world, d=args.degree)
    if world > 1:
        idx = lambda_round_robin(wl.points.re, wl.points.im, rank, world)
        wl.points = W.Points(np.ascontiguousarray(wl.points.re[idx]), np.ascontiguousarray(wl.points.im[idx]))
    return wl


def config(args, flush: bool):
    return {"workload": f"unit_disk_complex d={args.degree} (a_k uniform in unit disk, seed 1), "
                        f"{args.points} sphere-uniform points per GPU (one shared set of {args.points} x GPUs, "
                        f"split by lambda-sorted round-robin buckets), p=53",
            "degree": args.degree, "points_per_gpu": args.points, "p": 53,
            "l2": "flushed between steps (256 MiB write)" if flush else "not flushed"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def oracle_cpu_baseline(wl, n_sample: int, variants: bool = False):
    """Algorithm A_p restated by the CPU oracle on a bounded sample of points, on
    all host cores.  With variants, also on one core, and the plain FP64
    restatement of the window sums (hardware floats, the paper's p = 53 runs)
    on all cores and on one core."""
    import oracle
    t0 = time.perf_counter()
    pre = oracle.precondition(wl.coeffs, wl.p)
    t_pre = time.perf_counter() - t0
    zr, zi = wl.points.re[:n_sample], wl.points.im[:n_sample]
    oracle.fpe_eval(pre, zr[:16], zi[:16])  # warm-up (builds the C part)
    cores = oracle.num_threads()

    def timed(fn, n):
        t = time.perf_counter()
        fn(pre, zr[:n], zi[:n])
        return n / (time.perf_counter() - t)

    res = {"value": timed(oracle.fpe_eval, n_sample), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n_sample} of the workload's points (Alg. A_p windows + extended double-double "
                     f"window sums); preconditioning {t_pre:.2f} s not included"}
    if variants:
        n1 = max(64, n_sample // max(cores, 1))
        oracle.set_threads(1)
        try:
            res["single_core"] = {"value": timed(oracle.fpe_eval, n1), "cores": 1, "sample": f"{n1} points"}
            res["fp64_restatement_single_core"] = {
                "value": timed(oracle.fpe_eval_fp64, n1), "cores": 1, "sample": f"{n1} points",
                "kind": "plain FP64 CPU restatement of Alg. A_p (FP64 Horner over each window, z^l in "
                        "double-double)"}
        finally:
            oracle.set_threads(cores)
        res["fp64_restatement"] = {"value": timed(oracle.fpe_eval_fp64, n_sample), "cores": cores,
                                   "sample": f"{n_sample} points", "kind": "plain FP64 CPU restatement of Alg. A_p"}
    return res


def workload_legs(F, torch, st):
    """Evaluations/s on the benchmark's other workload shapes (the default
    configuration of fpe_eval; the d = 1000 one also with the tensor path off):
    d = 1000 unit square, 1/k! at d = 10^5, the Mandelbrot iterate at n = 20
    (d = 2^20, coefficients from workloads.mandelbrot_fast), sparse d = 2^22."""
    import workloads as W
    legs = {}
    for name, make in (("unit_square_d1000", lambda: W.unit_square_d1000()),
                       ("inverse_factorial_d1e5", lambda: W.inverse_factorial_d1e5(n_points=1 << 20)),
                       ("mandelbrot_n20", lambda: W.mandelbrot_real(20, n_points=1 << 20)),
                       ("sparse_d2pow22", lambda: W.sparse_d2pow22(n_points=1 << 20))):
        t0 = time.perf_counter()
        wl = make()
        t_gen = time.perf_counter() - t0
        t0 = time.perf_counter()
        P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im, wl.coeffs.e2, wl.p)
        t_pre = time.perf_counter() - t0
        zr = torch.from_numpy(wl.points.re).cuda()
        zi = None if wl.points.im is None else torch.from_numpy(wl.points.im).cuda()
        n = wl.points.n
        out = F.empty_out(n)
        nt = torch.empty(n, dtype=torch.int32, device="cuda")
        res = {"degree": wl.coeffs.n_coef - 1, "points": n, "precondition_ms": t_pre * 1e3,
               "generate_s": t_gen}
        for label, thr in (("default", None), ("tensor_off", 0)):
            if thr is not None and name != "unit_square_d1000":
                continue
            if thr is not None:
                F.fpe_set_tensor_path(P, thr)
            for _ in range(2):
                F.fpe_eval(P, zr, zi, out, nt)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            a.record(st)
            for _ in range(reps):
                F.fpe_eval(P, zr, zi, out, nt)
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            res[label] = {"evals_per_s": n / (ms * 1e-3), "ms_per_eval": ms,
                          "avg_kept_terms": float(nt.double().mean().item()),
                          "tensor_stats": F.fpe_tensor_stats(P)}
        F.fpe_sync(P)
        legs[name] = res
        del P, zr, zi, out, nt
    return legs


def batched_leg(F, torch, st):
    """4096 polynomials, degree log-uniform in [16, 2^16], log2|a_k| = s k + N(0,4),
    256 sphere points each, one fpe_batch_eval (FP64 p = 53 and FP32 p = 24)."""
    import workloads as W
    wls = W.batched_lognormal(n_poly=4096, pts_per_poly=256, seed=3)
    offs = np.concatenate([[0], np.cumsum([w.points.n for w in wls])]).astype(np.int64)
    zr = torch.from_numpy(np.concatenate([w.points.re for w in wls])).cuda()
    zi = torch.from_numpy(np.concatenate([w.points.im for w in wls])).cuda()
    res = {"polynomials": len(wls), "points": int(offs[-1]),
           "coefficients": int(sum(w.coeffs.n_coef for w in wls))}
    for name, p, flags in (("fp64", 53, 0), ("fp32", 24, F.FPE_FP32)):
        t0 = time.perf_counter()
        polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im, None, p, flags) for w in wls]
        res[f"{name}_precondition_s"] = time.perf_counter() - t0
        B = F.fpe_batch_create(polys, offs)
        res[f"{name}_tuning"] = F.fpe_batch_autotune(B, zr, zi)
        out = F.empty_out(B.n)
        F.fpe_batch_eval(B, zr, zi, out=out)
        F.fpe_batch_sync(B)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(5):
            F.fpe_batch_eval(B, zr, zi, out=out)
        b.record(st)
        torch.cuda.synchronize()
        res[f"{name}_evals_per_s"] = 5 * B.n / (a.elapsed_time(b) * 1e-3)
        # the same evaluation replayed from a captured CUDA graph
        s2 = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s2):
            F.fpe_batch_eval(B, zr, zi, out=out, stream=s2)
        g.replay()
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(5):
            g.replay()
        b.record(st)
        torch.cuda.synchronize()
        res[f"{name}_graph_evals_per_s"] = 5 * B.n / (a.elapsed_time(b) * 1e-3)
        del g, B, polys
    return res


def differentiation_leg(F, torch, st):
    """d = 2^18 unit-disk coefficients (+1e-3 noise), 2^20 sphere points: forward
    P, P', one Newton step, and the backward kernels (dL/dz, dL/da_k)."""
    import workloads as W
    wl, _, _ = W.differentiation_d2pow18()
    n = wl.points.n
    P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im, None, 53, F.FPE_WITH_DERIV)
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = torch.from_numpy(wl.points.im).cuda()
    g = torch.ones(n, dtype=torch.float64, device="cuda")
    ga_re = torch.zeros(wl.coeffs.n_coef, dtype=torch.float64, device="cuda")
    ga_im = torch.zeros_like(ga_re)
    out = F.empty_out(n)
    steps = {
        "forward_P": lambda: F.fpe_eval(P, zr, zi, out),
        "derivative_P1": lambda: F.fpe_eval_deriv(P, zr, zi, out),
        "newton_step": lambda: F.fpe_newton(P, zr, zi, out),
        "grad_points": lambda: F.fpe_grad_points(P, zr, zi, g, g),
        "grad_coeffs": lambda: F.fpe_grad_coeffs(P, zr, zi, g, g, ga_re, ga_im),
    }
    res = {"degree": wl.coeffs.n_coef - 1, "points": n}
    for name, fn in steps.items():
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        res[f"{name}_evals_per_s"] = n / (a.elapsed_time(b) * 1e-3)
    F.fpe_sync(P)
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args)
    n_sample = 4096
    steps = []
    base = None
    for i in range(args.warmup + args.steps):
        b = oracle_cpu_baseline(wl, n_sample)
        if i >= args.warmup:
            steps.append(b["value"])
        base = b
    v = float(np.median(steps))
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_sample / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, False), "cpu_baseline": base,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    import paper_2211_06320_gb300 as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    F._load()

    wl = workload(args, rank, world)
    n = wl.points.n
    t0 = time.perf_counter()
    P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im, None, 53)
    t_pre = time.perf_counter() - t0
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = torch.from_numpy(wl.points.im).cuda()
    out = F.empty_out(n)
    nterms = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    # launch parameters of the window sums picked by the library's autotuner on
    # this rank's points (before the timed region, like the preconditioning)
    t0 = time.perf_counter()
    tuning = F.fpe_autotune(P, zr, zi) if not args.no_tune else F.fpe_get_tuning(P)
    t_tune = time.perf_counter() - t0

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        F.fpe_eval(P, zr, zi, out, nterms)
    F.fpe_sync(P)
    # per-point work counts of this workload (same every step)
    nt = nterms.cpu().numpy().astype(np.int64)
    l, r, _ = F.fpe_get_windows(P, n)
    L = (r - l + 1).cpu().numpy()

    # timed region: K steps, L2 flushed between steps, each step's eval timed by events
    F.fpe_profile_reset()
    F.fpe_profile_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(st)
        F.fpe_eval(P, zr, zi, out, nterms)
        ev[i][1].record(st)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    F.fpe_profile_enable(False)
    F.fpe_sync(P)
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    t_dev = float(step_ms.sum()) / 1e3
    k_short, n_short = F.fpe_profile_read("k_sum_short")
    k_long, n_long = F.fpe_profile_read("k_sum_groups")
    k_fin, _ = F.fpe_profile_read("k_finalize_long")
    k_tc, n_tc = F.fpe_profile_read("k_tc_sum")
    k_all, launches = F.fpe_profile_read("")
    tcs = F.fpe_tensor_stats(P)
    if world > 1:
        t = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
    if world > 1:  # the shared point set's size: every rank's share was evaluated
        nt_all = torch.tensor([n], dtype=torch.int64, device="cuda")
        dist.all_reduce(nt_all)
        n_job = int(nt_all.item())
    else:
        n_job = n
    value = n_job * args.steps / t_dev

    # end to end through the C ABI with host buffers (pinned), copies inside the
    # timed region; every rank its own share, the slowest rank's time
    hz_r = torch.from_numpy(wl.points.re).pin_memory()
    hz_i = torch.from_numpy(wl.points.im).pin_memory()
    hout = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    for _ in range(2):
        F.host_eval_raw(P, hz_r.data_ptr(), hz_i.data_ptr(), n, hout.data_ptr())
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s = F.host_eval_raw(P, hz_r.data_ptr(), hz_i.data_ptr(), n, hout.data_ptr())
        assert s == 0
    dt = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    e2e = {"value": n_job * e2e_steps / dt, "unit": UNIT, "h2d_bytes_per_step": 16 * n_job,
           "d2h_bytes_per_step": 24 * n_job}

    extras = {}
    if rank == 0:
        # Which points took the tensor-core path: windows of at least min_window
        # terms (one coefficient piece here), minus any handed back (stats).
        tcp = F.fpe_get_tensor_path(P)
        tc_mask = (L >= tcp["min_window"]) if (tcp["min_window"] > 0 and tcp["pieces"] > 0) else np.zeros_like(L, bool)
        long_mask = (L > tuning["long_window"]) & ~tc_mask
        short_mask = ~long_mask & ~tc_mask
        # algorithmic FP64 flops of the kept terms: 8 per complex x complex term
        # (eq. complexityAlgo's Horner part)
        fl_short = 8.0 * float(nt[short_mask].sum())
        fl_long = 8.0 * float(nt[long_mask].sum())
        fl_tc_alg = 8.0 * float(nt[tc_mask].sum())
        fma_peak = F.fpe_measure_fma_peak(64, 5)
        fp64_peak_tflops = 2.0 * fma_peak / 1e12
        bf16_peak, bf16_src = measured_bf16_peak()
        # the tensor-core kernel's own work: an MMA sub-tile (8 blocks of 32 terms by a
        # tile's 128 point rows) is 4 k-steps x 10 tcgen05.mma, M = 128, K = 16,
        # N = 16 (10 - s) for Z' digit slice s: 2 x 128 x 64 x 880 flop of exact
        # 7-bit digit products
        fl_tc = float(tcs["subtiles"]) * TC_FLOPS_PER_SUBTILE
        kern = {"k_sum_short": (k_short / max(n_short, 1), fl_short),
                "k_sum_groups": (k_long / max(n_long, 1), fl_long),
                "k_tc_sum": (k_tc / max(n_tc, 1), fl_tc)}
        dom = max(kern, key=lambda k: kern[k][0])
        share = {k: (v[0] * args.steps) / max(k_all, 1e-9) for k, v in kern.items()}
        step_s = float(step_ms.mean()) * 1e-3
        fp64_equiv = {"algorithmic_flops_per_step": fl_short + fl_long + fl_tc_alg,
                      "achieved_tflops": (fl_short + fl_long + fl_tc_alg) / step_s / 1e12,
                      "fp64_peak_tflops": fp64_peak_tflops,
                      "frac_of_fp64_peak": (fl_short + fl_long + fl_tc_alg) / step_s / 1e12 / fp64_peak_tflops,
                      "note": "8 flop per kept complex term (the paper's count) over the whole step, against the "
                              "measured FP64 FMA peak; above 1 because the long windows run on the tensor cores"}

        def tensor_entry():
            ms, fl = kern["k_tc_sum"]
            traffic, traffic_note = measured_traffic("k_tc_sum")
            achieved = fl / max(ms * 1e-3, 1e-12) / 1e12
            return {"bound": "tensor", "kernel": "k_tc_sum", "achieved": achieved, "peak": bf16_peak,
                    "unit": "TFLOP/s", "frac": achieved / bf16_peak, "traffic": traffic,
                    "traffic_source": traffic_note, "peak_source": bf16_src, "share": share,
                    "flops_per_launch": fl, "launch_ms": ms,
                    "algorithmic_flops": "bf16 tensor flops of the exact digit products as issued: per MMA "
                                         "sub-tile 40 tcgen05.mma (M 128, K 16, N 16 (10 - s)), "
                                         "tensor_stats.subtiles x %.4g" % TC_FLOPS_PER_SUBTILE,
                    "method_work": {"flops_per_launch": fl_tc_alg,
                                    "tflops": fl_tc_alg / max(ms * 1e-3, 1e-12) / 1e12,
                                    "frac_of_fp64_peak": fl_tc_alg / max(ms * 1e-3, 1e-12) / 1e12 / fp64_peak_tflops,
                                    "note": "the paper's 8 flop per kept complex term of the points this kernel "
                                            "sums, per launch time, against the measured FP64 FMA peak"},
                    "tensor_stats": tcs}

        def fp64_entry(name):
            ms, fl = kern[name]
            traffic, traffic_note = measured_traffic(name)
            achieved = fl / max(ms * 1e-3, 1e-12) / 1e12
            return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": fp64_peak_tflops,
                    "unit": "TFLOP/s", "frac": achieved / fp64_peak_tflops, "traffic": traffic,
                    "traffic_source": traffic_note,
                    "peak_source": "measured: fpe_measure_fma_peak(64) on this GPU in this run (FP64 FMA x2)",
                    "share": share, "flops_per_launch": fl, "launch_ms": ms,
                    "algorithmic_flops": "8 per kept complex term (4 FMA: one complex multiply-add of "
                                         "Horner's scheme on G_p cap [l, r])",
                    "fma_issued_per_term": "4 at or above the peak term, 5 below it (blocks of four)"}

        roofline = tensor_entry() if dom == "k_tc_sum" else fp64_entry(dom)
        roofline["fp64_equivalent"] = fp64_equiv
        overlap = ("the FP64 window sums (caller's stream) and the tensor-core branch (the handle's second "
                   "stream) run at once and share the SMs, so each launch time spans the overlap: "
                   "achieved is the kernel's work over its own launch window, the shares sum above 1")
        if n_tc:
            roofline["overlap"] = overlap
        if dom != "k_tc_sum" and n_tc:
            extras["roofline_tensor_kernel"] = tensor_entry()
            extras["roofline_tensor_kernel"]["overlap"] = overlap
        extras["roofline"] = roofline
        extras["gpu_launches"] = int(launches)
        extras["avg_kept_terms"] = float(nt.mean())
        extras["avg_window"] = float(L.mean())
        extras["precondition_ms"] = t_pre * 1e3
        extras["tuning"] = dict(tuning, autotune_s=t_tune, autotuned=not args.no_tune)
        extras["wall_s_timed_region"] = wall

        extras["e2e"] = e2e

        if not args.no_extras:
            # GPU Horner baselines over all d+1 terms, one thread per point, on enough
            # points to occupy every SM (per-point work is fixed, so evaluations/s
            # do not depend on how many points are timed)
            for comp, m in ((False, 1 << 17), (True, 1 << 15)):
                sub_r, sub_i = zr[:m].contiguous(), zi[:m].contiguous()
                o2 = F.empty_out(m)
                F.fpe_horner(P, sub_r[:4096].contiguous(), sub_i[:4096].contiguous(), compensated=comp,
                             out=o2[:4096])
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                F.fpe_horner(P, sub_r, sub_i, compensated=comp, out=o2)
                b.record(st)
                torch.cuda.synchronize()
                sec = a.elapsed_time(b) * 1e-3
                key = "horner_compensated" if comp else "horner_plain"
                extras[key + "_evals_per_s"] = m / sec
                # the plain scheme's count: 8 flop per complex term, d + 1 terms per point
                fl = 8.0 * (args.degree + 1) * m
                # FP64 instructions each complex term issues: plain, 4 FMA and the two
                # multiplies of the coefficient's 2^-E scale; compensated, 4 TwoProd (2 each),
                # 4 TwoSum (6 each), 6 adds of the error terms, 4 FMA of the error recurrence
                # and the same 2 multiplies
                ins = 44 if comp else 6
                issue = ins * (args.degree + 1) * m / sec  # FP64 instructions per second
                extras[key + "_fp64"] = {"points": m, "seconds": sec, "flops_8_per_term": fl,
                                         "frac_of_fp64_peak": fl / sec / 1e12 / fp64_peak_tflops,
                                         "fp64_instructions_per_term": ins,
                                         "frac_of_fp64_issue": issue / (fp64_peak_tflops * 1e12 / 2.0)}
            # accuracy on a sample against the oracle's extended-precision Horner
            import oracle
            sample = np.unique(np.concatenate([np.arange(48), np.argsort(-L)[:16]]))
            ref, (Sm, Se), _ = oracle.horner_ref(wl.coeffs, wl.points.re[sample], wl.points.im[sample])
            got = out.cpu().numpy()[sample]
            ge = np.ascontiguousarray(got[:, 2]).view(np.int64)
            sc = lambda mm, ee: np.ldexp(mm, np.clip(ee - Se, -2000, 2000).astype(np.int32))
            err = np.hypot(sc(got[:, 0], ge) - sc(ref.re_hi, ref.e) - sc(ref.re_lo, ref.e),
                           sc(got[:, 1], ge) - sc(ref.im_hi, ref.e) - sc(ref.im_lo, ref.e)) / Sm
            extras["accuracy"] = {"max_err_over_S": float(err.max()), "tolerance": 2.0 ** -50,
                                  "sample_points": int(sample.size)}
            # FPE_ACCURATE throughput (compensated window sums)
            PA = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im, None, 53, F.FPE_ACCURATE)
            F.fpe_eval(PA, zr, zi, out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            F.fpe_eval(PA, zr, zi, out)
            b.record(st)
            torch.cuda.synchronize()
            extras["fpe_accurate_evals_per_s"] = n / (a.elapsed_time(b) * 1e-3)
            # FP32 mode (p = 24: windows from T = 24 + s(d) + 3, FP32 coefficients and Horner)
            P32 = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im, None, 24, F.FPE_FP32)
            nt32 = torch.empty(n, dtype=torch.int32, device="cuda")
            F.fpe_eval(P32, zr, zi, out, nt32)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            F.fpe_eval(P32, zr, zi, out, nt32)
            b.record(st)
            torch.cuda.synchronize()
            extras["fpe_fp32_p24_evals_per_s"] = n / (a.elapsed_time(b) * 1e-3)
            extras["fpe_fp32_p24_avg_kept_terms"] = float(nt32.double().mean().item())
            extras["cpu_baseline"] = oracle_cpu_baseline(wl, 4096, variants=True)
            extras["workloads"] = workload_legs(F, torch, st)
            extras["batched"] = batched_leg(F, torch, st)
            extras["differentiation"] = differentiation_leg(F, torch, st)

        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config(args, True), "clocks": clk}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
