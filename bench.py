"""Benchmark: PAM sweeps/s of trace-regularized FCTN completion on GB300.

One step = one PAM sweep (every factor update of Eqs. 4-9 in the order
1..N, then the X update of Eq. 10) over the full workload, inputs resident
in device memory.  Default workload: 256 x 256 x 31 x 8 (a multispectral
sequence), all FCTN ranks 6, Bernoulli(0.1) mask, lambda = 0.01, rho = 0.1,
TF32 tensor-core contractions (the mixed-precision path); `precision_modes`
times the same workload in FP32 (CUDA cores), TF32 and BF16 and reports the
final PSNR of each.  X is 65 MB, smaller than L2, so L2 is flushed (a 256 MB
write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c4] [--precision tf32]

Under torchrun every rank runs an independent replica on its own GPU (the
method has no data-path exchange: replicas only), value = all ranks' sweeps /
max-over-ranks time.  `--impl reference` times the FP64 CPU oracle on the same
workload (one oracle sweep per step) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_22506_gb300 import synth  # noqa: E402

METRIC = "PAM sweeps/s & time-to-tol, mixed-prec+served vs plain FP32 on 1 GB300; p50/p99"
UNIT = "sweeps/s"
DESC = {
    "c1": "30x30x10 FCTN rank 3, SR 0.3, FP64 parity workload",
    "c2": "256x256x31 multispectral-shaped, FCTN rank 8, SR 0.1, noise 0.01",
    "c3": "144x176x3x50 colour-video-shaped, FCTN rank 6 (3 on the colour mode), SR 0.05",
    "c4": "256x256x31x8 multispectral sequence, FCTN rank 6, SR 0.1",
}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # CUDA-core FP32 at the maximum SM clock
SM_FP32_TFLOPS = 128 * 2 * 2.07e9 / 1e12           # one SM (single-CTA kernels)


def eig_sms(s):
    """SMs of the FP32 Gram eigensolver: one CTA up to s = 64, else a cluster of
    4-8 CTAs with T tables each, m = 8 CL T >= s padded least (as the library)."""
    if s <= 64:
        return 1, "k_eig3 (one CTA)"
    need = (s + 7) // 8
    best = None
    for cl in range(8, 3, -1):
        t = -(-need // cl)
        if best is None or 8 * cl * t < best[0]:
            best = (8 * cl * t, cl)
    return best[1], f"k_eigc (cluster of {best[1]} CTAs, m = {best[0]})"
# Kernel behind each profiler class of the head-mode route, and its bound.
CLASS_KERNEL = {
    "gram": ("k_tg_gemm (X_(1) M_1^T, X_(1)^T A_(1))", "hbm"),
    "xupdate": ("k_tg_gemm (F^T = M_1^T A_(1)^T, Eq. 10 epilogue)", "hbm"),
    "eig": ("k_chol_factor (one CTA per distinct shift of Eq. 6)", "chol"),
    "env": ("k_sgemm (factor Grams and their chains)", "alu"),
    "rhs2": ("k_sgemm (right-hand sides 2..N from Z)", "alu"),
    "merged": ("k_sgemm (M_1) + operand copies", "alu"),
    "solve": ("k_bgemm (Q^T R, Q W with the L_k basis)", "alu"),
    "subst": ("k_chol_subst (triangular substitutions, one CTA per row group)", "alu"),
    "resid": ("k_resid_df (Eq. 5 residual, double-float A G)", "alu"),
    "eigaux": ("k_mm_small, k_first_order, k_eig_apply", "alu"),
    "reduce": ("k_tg_reduce, k_finish_rhs", "hbm"),
    "misc": ("k_trace, k_finalize, copies", "hbm"),
}
# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of the
# current kernel on this workload (profiles/); absent when not captured since
# the kernel last changed.
TRAFFIC = {
    ("c4", "tf32", "eig"): (0.22e6, "dram__bytes_read.sum + dram__bytes_write.sum of one k_chol_factor launch (129 CTAs), "
                                    "ncu --set full on the 256x256x31x8 TF32 sweep (profiles/chol_solve_256x256x31x8_tf32.md)"),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th is not None:
            self.th.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def max_over_ranks(total_ms, dist, device=None):
    """Timed-region length of the slowest rank (every rank gets it)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, world_size, total_ms):
    """Whole-job sweeps/s: every rank ran `steps` sweeps of its own replica."""
    return steps * world_size / (total_ms / 1e3)


def gpu_inputs(F, name):
    """Workload inputs; the ground-truth contraction runs on the library's own path."""
    w = synth.WORKLOADS[name]
    dims = tuple(w["dims"])

    def contract(fs):
        R = synth.rank_matrix(dims, w["r"], w["cap"])
        p = F.make_params(dims, R, precision="fp64", reuse=False)
        h = F.fctn_create(p)
        try:
            F.fctn_set_factors(h, [np.ascontiguousarray(a) for a in fs])
            out = np.empty(dims, dtype=np.float64)
            F.fctn_contract(h, out)
        finally:
            F.fctn_destroy(h)
        return out

    return synth.workload_inputs(name, contract)


def sweep_floor_bytes(dims, R):
    """Minimal HBM bytes of one sweep: N + 1 passes over X in FP32 (N right-hand
    sides and the X update), one write of X, one mask bit per element."""
    P = int(np.prod(dims))
    return (len(dims) + 2) * 4.0 * P + P / 8.0


# the M_1 chain and the right-hand-side chains run on the tensor cores in the
# TF32 / BF16 precisions: bound by the gathered operand bytes
CLASS_KERNEL_TC = {
    "rhs2": ("k_tcc (right-hand sides 2..N from Z; tcgen05 TF32, operands gathered through offset tables)", "hbm"),
    "merged": ("k_tcc (M_1 chain; tcgen05 TF32) + operand copies", "hbm"),
}


def class_roofline(cls, prof, peaks, peak_src, precision, svals, eig_sweeps, dims=None):
    """Achieved rate of one kernel class (one kernel per launch) against its roof."""
    kernel, bound = CLASS_KERNEL.get(cls, (cls, "hbm"))
    if precision in ("tf32", "bf16") and cls in CLASS_KERNEL_TC:
        kernel, bound = CLASS_KERNEL_TC[cls]
    n = max(prof["launches"], 1)
    avg_s = prof["ms"] / n / 1e3
    if bound == "chol" and eig_sweeps == 0:
        # one CTA per distinct shift (floor(I / 2) + 1 of them), s^3 / 3 flops
        # each (Cholesky of an s x s matrix); every CTA does the same work, so
        # the per-CTA rate against one SM's FP32 rate is the fraction
        groups = [I // 2 + 1 for I in dims]
        flops = float(np.mean([g * sv ** 3 / 3.0 for g, sv in zip(groups, svals)]))
        sms = float(np.mean([min(g, 152) for g in groups]))
        ach = flops / avg_s / 1e12
        peak = sms * SM_FP32_TFLOPS
        return dict(kernel=kernel, bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_source=f"derived: {sms:.1f} SMs (one CTA per shift, mean over the factors) x 128 FP32 "
                                "lanes x 2 x 2.07 GHz",
                    flops_per_launch=flops)
    if bound in ("alu1", "chol"):  # the SMs the eigensolver runs on; two-sided Jacobi on B and V^T, 9 s^3 flops per sweep
        flops = float(np.mean([9.0 * sv ** 3 for sv in svals])) * max(eig_sweeps, 1)
        sms, kname = eig_sms(max(svals))
        ach = flops / avg_s / 1e12
        peak = sms * SM_FP32_TFLOPS
        return dict(kernel=kname, bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_source=f"derived: {sms} SM(s) x 128 FP32 lanes x 2 x 2.07 GHz",
                    flops_per_launch=flops)
    if bound == "alu":
        ach = prof["flops"] / n / avg_s / 1e12
        return dict(kernel=kernel, bound="alu", achieved=ach, peak=FP32_PEAK_TFLOPS, unit="TFLOP/s",
                    frac=ach / FP32_PEAK_TFLOPS, peak_source="derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                    flops_per_launch=prof["flops"] / n)
    ach = prof["bytes"] / n / avg_s / 1e9
    out = dict(kernel=kernel, bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
               frac=ach / peaks["hbm_gbs"], peak_source=f"{peak_src} HBM copy bandwidth",
               bytes_per_launch=prof["bytes"] / n)
    if prof["flops"] > 0 and precision in ("tf32", "bf16"):
        tpk = peaks["bf16_tflops"] * (0.5 if precision == "tf32" else 1.0)
        out["tensor_tflops"] = prof["flops"] / n / avg_s / 1e12
        out["tensor_frac"] = out["tensor_tflops"] / tpk
        out["tensor_peak_source"] = f"{peak_src} dense BF16" + (" x nominal TF32/BF16 0.5" if precision == "tf32" else "")
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2510_22506_gb300 import fctn as F

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = args.workload
    w = synth.WORKLOADS[name]
    truth, Y, mask, init, R = gpu_inputs(F, name)
    N = len(w["dims"])
    precision = args.precision
    p = F.make_params(Y.shape, R, lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO, precision=precision,
                      reuse=True, order_policy="plain")
    dt = F.elem_dtype(p)
    stream = torch.cuda.Stream(device=dev)
    Yd = torch.from_numpy(np.ascontiguousarray(Y.astype(dt))).to(dev)
    Md = torch.from_numpy(mask.astype(np.uint8)).to(dev)
    initd = [torch.from_numpy(np.ascontiguousarray(a.astype(dt))).to(dev) for a in init]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    torch.cuda.synchronize()
    # launch shapes from libfctn's autotuner (probe handles on the same
    # inputs), before the timed region
    tune = None
    if not args.no_tune:
        best, tms = F.fctn_autotune_tiles(p, Yd, Md, initd, sweeps=3, stream=stream)
        p.tile_code = best
        tune = {"tile_code": best, "sweep_ms": {str(c): round(v, 4) for c, v in tms.items()}}
    h = F.fctn_create(p, stream)
    try:
        F.fctn_set_data(h, Yd, Md)
        F.fctn_set_factors(h, initd)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                F.fctn_pam_sweep(h, 1, want_stats=False)
                flush.zero_()
        torch.cuda.synchronize()
        # ---- timed region: K sweeps, L2 flushed between them (outside the events)
        clocks = ClockSampler(local)
        clocks.start()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = F.fctn_launch_count(h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                ev[i][0].record(stream)
                F.fctn_pam_sweep(h, 1, want_stats=False)
                ev[i][1].record(stream)
                flush.zero_()
        torch.cuda.synchronize()
        launches = F.fctn_launch_count(h) - l0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = float(sum(step_ms))
        if ws > 1:
            total_ms = max_over_ranks(total_ms, dist, dev)
            dist.barrier()
        clk = clocks.stop()
        st = F.fctn_pam_sweep(h, 0)
        # ---- per-class device time: CUDA events around every launch of one
        # class (eager sweeps, one class at a time), 2 sweeps per class
        per_class = {}
        with torch.cuda.stream(stream):
            for cls in F.KC:
                F.fctn_profile(h, cls)
                for _ in range(2):
                    F.fctn_pam_sweep(h, 1, want_stats=False)
                    flush.zero_()
                per_class[cls] = F.fctn_profile_read(h)
            F.fctn_profile(h, None)
        st2 = F.fctn_pam_sweep(h, 0)
        # ---- end to end through the C ABI with host buffers
        e2e_sweeps = 10

        def pinned(a):  # page-locked host copy (NumPy view of a pinned torch tensor)
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

        Yh = pinned(Y.astype(dt))
        Mh = pinned(mask.astype(np.uint8))
        inith = [pinned(a.astype(dt)) for a in init]
        Xh = pinned(np.empty(Y.shape, dtype=dt))
        e2e_times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.fctn_set_data(h, Yh, Mh)
            F.fctn_set_factors(h, inith)
            F.fctn_pam_sweep(h, e2e_sweeps, want_stats=False)
            F.fctn_get_X(h, Xh)
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = min(e2e_times)
        h2d = Yh.nbytes + Mh.nbytes + sum(a.nbytes for a in inith)
        d2h = Xh.nbytes
    finally:
        F.fctn_destroy(h)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    value = job_value(args.steps, ws, total_ms)
    peaks, peak_src = load_peaks()
    svals = [int(np.prod([R[min(k, t), max(k, t)] for t in range(N) if t != k])) for k in range(N)]
    eig_sw = int(st2["eig_sweeps"])
    rows = {c: class_roofline(c, v, peaks, peak_src, precision, svals, eig_sw, dims=w["dims"])
            for c, v in per_class.items() if v["launches"] > 0}
    for c, v in per_class.items():
        if c in rows:
            rows[c].update(ms_per_sweep=v["ms"] / 2, launches_per_sweep=v["launches"] / 2,
                           avg_launch_us=v["ms"] / max(v["launches"], 1) * 1e3)
    dom = max(rows, key=lambda c: per_class[c]["ms"])
    roof = dict(rows[dom])
    roof["kernel_class"] = dom
    tr = TRAFFIC.get((name, precision, dom))
    roof["traffic"] = tr[0] if tr else None
    roof["traffic_of"] = tr[1] if tr else "not captured for the current kernel"
    roof["measured"] = "CUDA events around each launch of the class on the handle's stream, 2 eager sweeps"
    floor_b = sweep_floor_bytes(w["dims"], R)
    ms = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16", "fp64": "f64"}[precision], "data": "synthetic",
        "config": {"workload": f"{name}: {DESC[name]}", "dims": list(w["dims"]), "rank": w["r"], "sampling": w["p"],
                   "precision": precision, "reuse": True, "order_policy": "plain", "lambda": synth.LAMBDA,
                   "delta": synth.DELTA, "rho": synth.RHO, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{ws}", "graphs": True,
                   "autotune": tune if tune else "off (built-in launch shapes)"},
        "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms),
        "rel_change_last": st["rel_change"], "eig_sweeps_last": st["eig_sweeps"],
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "kernel_classes": rows,
        "sweep_floor": {"bytes": floor_b, "floor_us": floor_b / (peaks["hbm_gbs"] * 1e9) * 1e6,
                        "frac": floor_b / (peaks["hbm_gbs"] * 1e9) / (ms / 1e3),
                        "what": "(N + 2) FP32 passes over X + 1 mask bit per element, at the measured HBM copy rate"},
        "e2e": {"value": e2e_sweeps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "step": f"set_data + set_factors from pinned host buffers, {e2e_sweeps} sweeps, X back to pinned host memory"},
    }
    if ws == 1 and not args.no_extras:
        xs = min(args.steps, 20)  # timed sweeps of the comparison runs
        line["solve_routes"] = solve_routes(F, Y, mask, init, R, precision, xs)
        line["precision_modes"] = precision_modes(F, name, truth, Y, mask, init, R, xs, tune=not args.no_tune)
        if name != "c2":
            line["secondary_c2"] = precision_modes(F, "c2", *gpu_inputs(F, "c2"), xs, quality_sweeps=0,
                                                   tune=not args.no_tune)
        line["rank_growth"] = rank_growth_run(F, "c2", *gpu_inputs(F, "c2"))
        line["serving"] = serving_mix(args.serve_jobs, tune=not args.no_tune)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def solve_routes(F, Y, mask, init, R, precision, steps, warm=5):
    """ms per sweep with each solve of Eq. 5 (FCTN_SOLVE_CHOL, the default
    here, and FCTN_SOLVE_EIG, Eq. 8 through the Jacobi eigendecomposition),
    graphs, L2 flushed between sweeps, after `warm` untimed sweeps."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    Y32, M8 = np.ascontiguousarray(Y.astype(np.float32)), mask.astype(np.uint8)
    init32 = [np.ascontiguousarray(a.astype(np.float32)) for a in init]
    out = {}
    for m in ("chol", "eig"):
        p = F.make_params(Y.shape, R, lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO, precision=precision,
                          order_policy="plain", solve_method=m)
        st = torch.cuda.Stream()
        h = F.fctn_create(p, st)
        try:
            F.fctn_set_data(h, Y32, M8)
            F.fctn_set_factors(h, init32)
            F.fctn_pam_sweep(h, warm, want_stats=False)
            tot = 0.0
            with torch.cuda.stream(st):
                for _ in range(steps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    F.fctn_pam_sweep(h, 1, want_stats=False)
                    b.record(st)
                    flush.zero_()
                    b.synchronize()
                    tot += a.elapsed_time(b)
            out[m] = {"ms_per_sweep": tot / steps, "eig_sweeps_last": F.fctn_pam_sweep(h, 0)["eig_sweeps"]}
        finally:
            F.fctn_destroy(h)
    return out


def precision_modes(F, name, truth, Y, mask, init, R, steps, quality_sweeps=100, tol=1e-4, max_sweeps=500,
                    tune=True):
    """The same workload in every precision (plain order, reuse): sweeps/s
    (graphs, L2 flushed between sweeps), PSNR / SSIM against the truth
    (Sec. 4, computed by libfctn) after `quality_sweeps` sweeps from the same
    start, and time to tolerance (fctn_complete to rel < tol, at most
    max_sweeps sweeps, wall clock) with its final PSNR."""
    import torch
    out, quality, ttt, tuned = {}, {}, {}, {}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    truth32 = np.ascontiguousarray(truth.astype(np.float32))
    Y32, M8 = np.ascontiguousarray(Y.astype(np.float32)), mask.astype(np.uint8)
    init32 = [np.ascontiguousarray(a.astype(np.float32)) for a in init]
    for prec in ("fp32", "tf32", "bf16"):
        # the reduced precisions finish in FP32 once rel_change <= 1e-3: the
        # tensor-core products' rounding alone keeps it near 4e-4 on 256x256x31x8
        p = F.make_params(Y.shape, R, lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO, precision=prec,
                          order_policy="plain", finish_fp32_at=1e-3 if prec != "fp32" else 0.0)
        st = torch.cuda.Stream()
        if tune:
            p.tile_code, _ = F.fctn_autotune_tiles(p, Y32, M8, init32, sweeps=3, stream=st)
            tuned[prec] = p.tile_code
        h = F.fctn_create(p, st)
        try:
            F.fctn_set_data(h, Y32, M8)
            F.fctn_set_factors(h, init32)
            tot = 0.0
            with torch.cuda.stream(st):
                for i in range(steps + 3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    F.fctn_pam_sweep(h, 1, want_stats=False)
                    b.record(st)
                    flush.zero_()
                    b.synchronize()
                    if i >= 3:
                        tot += a.elapsed_time(b)
            out[prec] = steps / (tot / 1e3)
            if quality_sweeps > 0:
                F.fctn_pam_sweep(h, max(quality_sweeps - steps - 3, 0), want_stats=False)
                ps, ss = F.fctn_quality(h, truth32)
                quality[prec] = {"psnr_db": ps, "ssim": ss}
                # time to tolerance from the same start
                F.fctn_set_data(h, Y32, M8)
                F.fctn_set_factors(h, init32)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = F.fctn_complete(h, tol, max_sweeps)
                wall = time.perf_counter() - t0
                ps, ss = F.fctn_quality(h, truth32)
                ttt[prec] = {"sweeps": r["t"], "wall_s": wall, "rel_change": r["rel_change"],
                             "converged": bool(r["converged"]), "psnr_db": ps, "ssim": ss}
        finally:
            F.fctn_destroy(h)
    res = {"unit": UNIT, "sweeps_per_s": out, "workload": name, "order_policy": "plain",
           "finish_fp32_at": 1e-3, "tile_code_autotuned": tuned or "off"}
    if quality_sweeps > 0:
        res.update({"quality_after_sweeps": max(quality_sweeps, steps + 3), "quality": quality,
                    "time_to_tol": {"tol": tol, "max_sweeps": max_sweeps, **ttt}})
    return res


def rank_growth_run(F, name, truth, Y, mask, init, R, grow_every=5, tol=1e-4, max_sweeps=150):
    """Plain FP32 to rel < tol (or max_sweeps) with fixed ranks R, and with the
    ranks grown from one to R (growth.complete_with_growth); wall time, sweeps,
    PSNR and SSIM of each."""
    import torch
    from paper_2510_22506_gb300 import growth
    N = Y.ndim
    kw = dict(lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO)
    truth32 = np.ascontiguousarray(truth.astype(np.float32))
    out = {"workload": name, "tol": tol, "max_sweeps": max_sweeps}
    p = F.make_params(Y.shape, R, precision="fp32", **kw)
    h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, np.ascontiguousarray(Y.astype(np.float32)), mask.astype(np.uint8))
        F.fctn_set_factors(h, [np.ascontiguousarray(a.astype(np.float32)) for a in init])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = F.fctn_complete(h, tol, max_sweeps)
        wall = time.perf_counter() - t0
        ps, ss = F.fctn_quality(h, truth32)
        out["fixed_ranks"] = {"sweeps": st["t"], "wall_s": wall, "rel_change": st["rel_change"], "psnr_db": ps,
                              "ssim": ss}
    finally:
        F.fctn_destroy(h)
    init1 = synth.init_factors(Y.shape, np.ones((N, N), dtype=int), 3900)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, hist = growth.complete_with_growth(Y, mask, init1, R, grow_every, 0.1, 4242, tol, max_sweeps,
                                          precision="fp32", **kw)
    try:
        wall = time.perf_counter() - t0
        ps, ss = F.fctn_quality(h, truth32)
        out["grown_from_one"] = {"grow_every": grow_every, "sweeps": len(hist), "wall_s": wall,
                                 "rel_change": hist[-1]["rel_change"], "psnr_db": ps, "ssim": ss}
    finally:
        F.fctn_destroy(h)
    return out


def serving_mix(n_jobs, tune=True, precision="tf32"):
    """Serving mix (Poisson 20 jobs/s, seeded; shapes 64x64x16, 128x128x31,
    144x176x3x20, 256x256x31; ranks {3,4,6}; SR {0.05,0.1,0.2}; to rel < 1e-4,
    cap 500): served (continuous batching, same-shape sweeps grouped into one
    graph per class) in the mixed precision vs the same arrivals served one
    job at a time in plain FP32; latency (arrival -> result) and time to
    tolerance p50 / p99, jobs/s, and the mean final PSNR of each arm."""
    from paper_2510_22506_gb300 import serve as S
    jobs = S.mix_jobs(n_jobs, seed=5000, rate=20.0)
    tuner = S.TuneCache().fill(jobs, precision) if tune else None
    served = S.run_mix(jobs, precision=precision, tol=1e-4, max_sweeps=500, max_jobs=64, tuner=tuner, group=True)
    seq = S.run_sequential(jobs, precision="fp32", tol=1e-4, max_sweeps=500)
    keys = ("jobs", "failed", "wall_s", "jobs_per_s", "sweeps", "sweeps_per_s", "latency_p50_s", "latency_p99_s",
            "ttt_p50_s", "ttt_p99_s", "psnr_mean_db", "group_launches", "group_captures")
    arrival_rate = n_jobs / max(j["arrival"] for j in jobs)
    return {f"served_{precision}": {k: served.get(k) for k in keys},
            "sequential_fp32": {k: seq.get(k) for k in keys if k in seq},
            "jobs_per_s_ratio": served["jobs_per_s"] / seq["jobs_per_s"],
            "arrival_rate_jobs_per_s": arrival_rate,
            "served_sustains_arrivals": served["jobs_per_s"] >= 0.95 * arrival_rate,
            "autotune": ({"classes": len(tuner.table), "tune_s": round(tuner.tune_s, 3),
                          "choices": sorted(set(tuner.table.values()))} if tuner else "off")}


def oracle_setup(name):
    from oracle import fctn_oracle as O
    truth, Y, mask, init, R = synth.workload_inputs(name, O.fctn_full)
    N = Y.ndim
    prob = O.Problem(dims=Y.shape, R=R, lam=(synth.LAMBDA,) * N, delta=(synth.DELTA,) * N, rho=synth.RHO)
    return O, O.init_state(Y, mask, init), prob


def cpu_baseline(name, budget_s=15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample."""
    O, st, prob = oracle_setup(name)
    O.pam_sweep(st, prob, policy="plain")  # warm-up
    n, t0 = 0, time.perf_counter()
    while True:
        O.pam_sweep(st, prob, policy="plain")
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full sweeps of workload {name} after one warm-up sweep ({el:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    O, st, prob = oracle_setup(args.workload)
    # bounded sample: one untimed sweep at most, then full sweeps until K are
    # done or the time budget is spent (a 256x256x31x8 sweep takes seconds)
    for _ in range(min(args.warmup, 1)):
        O.pam_sweep(st, prob, policy="plain")
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (done == 0 or time.perf_counter() - t0 < args.ref_budget):
        O.pam_sweep(st, prob, policy="plain")
        done += 1
    el = time.perf_counter() - t0
    value = done / el
    w = synth.WORKLOADS[args.workload]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": done,
        "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {DESC[args.workload]}", "dims": list(w["dims"]), "rank": w["r"],
                   "sampling": w["p"], "precision": "fp64 (CPU oracle)", "reuse": True,
                   "order_policy": "plain", "lambda": synth.LAMBDA, "delta": synth.DELTA, "rho": synth.RHO},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{done} full sweeps of workload {args.workload} (one per step, at most "
                                   f"{args.steps} or {args.ref_budget:.0f} s) after {min(args.warmup, 1)} untimed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(DESC))
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the precision and serving comparisons")
    ap.add_argument("--no-tune", action="store_true", help="built-in launch shape instead of the autotuner's")
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--ref-budget", type=float, default=60.0, help="seconds of timed oracle sweeps (reference arm)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
