"""Throughput of the hypergradient hot path on the 64-pair batch workload.

One step = one outer iteration over the batch (64 training pairs of uneven sizes, FoE with
16 5x5 filters): warm-started lower solve (L-BFGS), recycle refresh (by default the inner variant
of eq. (3.4), projected with the previous system's Hessian through its CG Lanczos record),
warm-started recycled-CG
Hessian solve, J w contraction, then an Adam update of theta (Section 5.2).  The metric is
hypergradients per second at a stopping tolerance that keeps every hypergradient within 1e-4
relative error of a tight reference solve (checked after the timed region and reported).

Arms
  default            the CUDA path (libbl), recycled CG with the chosen strategy; the same run
                     also times plain CG on the same sequence, warm-started and cold-started.
  --impl reference   the FP64 CPU checker on a bounded sample of the workload (host cores).

Other workloads: --workload inpaint (1024 pairs of 28 x 28, Section 5.1's shape) and
--workload deconv --method minres (512 pairs of 64 x 64, phi = log(1 + s^2), Section 5.2's
shape); --rtol sets the residual tolerance, --no-graph runs both loops host-polled (profilers).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own batch (weak scaling) and the mean
hypergradient is all-reduced once per step before the shared theta update.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

S_RECYCLE = 16         # recycle dimension of the 64-pair batch (30 for the inpainting batch)
MAX_BASIS = 32
RTOL = 1e-4            # residual stopping tolerance (relative to ||g||)
INPAINT_RTOL = 1e-5
DECONV_RTOL = 1e-5
LOWER_GTOL = 1e-5      # lower-level gradient tolerance (relative to ||grad Phi(0)||)
ADAM_LR = 1e-2
FP32_FMA_LANES = 152 * 128   # GB300: 152 SMs x 128 FP32 lanes
# DRAM bytes (read + write) per pixel of one fused Hessian action with the recycled-CG dots over
# 16 recycle columns, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum on the
# first 16 pairs of the batch: 179.3 MB for 1,306,624 px; summary in
# profiles/hvp_k_foe_stencil_f5_batch16.md), scaled to a launch by the pixels it processes.
HVP_DRAM_BYTES_PER_PIXEL = 137.2


def hvp_flops_per_pixel(n_filters, f, rb, masked=False):
    """Algorithmic FP32 flops of one Hessian action per pixel (fields variant):
    per filter K v (2 T), times d_j (1), K^T (2 T); blur A A v separable (4 passes x (2 r_b + 1)
    FMA = 8 (2 r_b + 1) flop), or for inpainting the mask product (2); l2 term and sum (2)."""
    T = f * f
    return n_filters * (4 * T + 1) + (2 if masked else 8 * (2 * rb + 1)) + 2


def hvp_bytes_per_pixel(n_filters, esz=4, masked=False):
    """Algorithmic HBM bytes of one Hessian action per pixel: v in, H v out, N fields d_j in (and
    the 1-byte mask for inpainting)."""
    return (2 + n_filters) * esz + (1 if masked else 0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bl_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# Workloads

def workload_rtol(name):
    return {"inpaint": INPAINT_RTOL, "deconv": DECONV_RTOL}.get(name, RTOL)


def make_workload(name, replica=0):
    """(workload, recycle dimension, description) for --workload.  The residual tolerance that
    keeps every hypergradient within 1e-4 is RTOL for the batch, INPAINT_RTOL for the inpainting
    pairs (70 % unmeasured pixels make their Hessians ill-conditioned: rtol 1e-4 left errors of
    2-3e-4) and DECONV_RTOL for the 64x64 deconvolution pairs (rtol 1e-4 left 1.1-1.4e-4)."""
    from paper_2412_08264_gb300 import synth
    if name == "inpaint":
        wl = synth.inpaint_batch(seed=replica)
        return wl, 30, (f"inpaint1024x28_n3f5: {len(wl.pairs)} pairs of 28x28, 30 % of pixels measured, "
                        f"noise 0.1, 3 5x5 filters, phi = s^2, p={wl.n_params}")
    if name == "deconv":
        wl = synth.deconv_batch(seed=replica)
        return wl, 16, (f"deconv512x64_n24f5: {len(wl.pairs)} pairs of 64x64, 9x9 blur sigma 3, noise 0.08, "
                        f"24 5x5 DCT-initialised filters, phi = log(1 + s^2), p={wl.n_params}")
    wl = synth.batch_64(replica=replica)
    return wl, S_RECYCLE, None


# ---------------------------------------------------------------------------------------------
# GPU arm

def gpu_arm(args, rank, world, dist):
    import torch
    from paper_2412_08264_gb300 import api, synth
    from paper_2412_08264_gb300.parallel import allreduce_mean
    from paper_2412_08264_gb300.strategy import parse

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl, s_rec, wdesc = make_workload(args.workload, replica=rank)
    rtol = args.rtol or workload_rtol(args.workload)
    if args.pairs and args.pairs < len(wl.pairs):
        wl.pairs, wl.x_star, wl.noise = wl.pairs[:args.pairs], wl.x_star[:args.pairs], wl.noise[:args.pairs]
    K = len(wl.pairs)
    xs_h = torch.tensor(np.concatenate([x.ravel() for x in wl.x_star]), dtype=torch.float32).pin_memory()
    nz_h = torch.tensor(np.concatenate([x.ravel() for x in wl.noise]), dtype=torch.float32).pin_memory()
    xs = xs_h.to(dev)
    P0 = api.from_workload(wl, xs, xs)
    if any(m is not None for m in wl.masks):
        y = P0.forward(xs + nz_h.to(dev))     # inpainting: noisy values at the measured pixels only
    else:
        y = P0.forward(xs) + nz_h.to(dev)
    del P0
    y_h = y.cpu().pin_memory()
    n_pix = xs.numel()
    strategy = parse(args.strategy)

    def run(strat, steps, warmup, e2e=False, validate=False, profile_range=False, prof_steps=0, warm=True):
        P = api.from_workload(wl, y, xs, max_recycle=s_rec, max_basis=args.max_basis)
        y_d = torch.empty_like(y)
        xs_d = torch.empty_like(xs)
        theta = wl.theta0.copy()
        theta_d = torch.tensor(theta, dtype=torch.float64, device=dev)
        m = np.zeros_like(theta)
        v2 = np.zeros_like(theta)
        xhat = P.zeros()
        w = P.zeros()
        stream = torch.cuda.current_stream(dev)
        iters = []
        hg_prev = None
        state = {"t": 0}

        def step(i, record):
            nonlocal theta, m, v2, hg_prev
            if e2e:
                y_d.copy_(y_h, non_blocking=True)
                xs_d.copy_(xs_h, non_blocking=True)
                P.set_data(y_d, xs_d)
            P.lower_solve(theta_d, xhat, gtol=LOWER_GTOL, relative=True, max_iters=2000, allow_noconv=True,
                          graph=args.graph)
            if strat.recycles and state["t"] > 0:
                P.ritz_update(strat, s_rec, variant=args.refresh)
            info = P.hessian_solve(w, recycle=strat.recycles, nsc=strat.nsc, tol=rtol, relative=True, maxit=3000,
                                   store_basis=(("lanczos" if args.refresh == "inner" else True)
                                                if strat.recycles else False), warm_start=warm,
                                   nsc_scale=None if hg_prev is None else [hg_prev] * K, allow_noconv=True,
                                   method=args.method, graph=args.graph)
            mean, per = P.hypergrad(w, per_pair=True)
            if world > 1:
                mean = allreduce_mean(mean, K)
            g = mean.cpu().numpy()                       # the step's result, read back every step
            hg_prev = float(np.linalg.norm(g))
            # Adam (Section 5.2: fixed step length 1e-2)
            state["t"] += 1
            t = state["t"]
            m = 0.9 * m + 0.1 * g
            v2 = 0.999 * v2 + 0.001 * g * g
            theta = theta - ADAM_LR * (m / (1 - 0.9 ** t)) / (np.sqrt(v2 / (1 - 0.999 ** t)) + 1e-8)
            theta_d.copy_(torch.from_numpy(theta), non_blocking=False)
            if record:
                iters.append([d["iters"] for d in info])
            return per

        for i in range(warmup):
            step(i, False)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = Clocks(dev.index)
        clocks.start()
        launches0 = P.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if profile_range:
            torch.cuda.profiler.start()
        ev0.record(stream)
        per = None
        for i in range(steps):
            per = step(i, True)
        ev1.record(stream)
        torch.cuda.synchronize()
        if profile_range:
            torch.cuda.profiler.stop()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        launches = P.launch_count() - launches0
        graph_used = P.graph_used()
        ck = clocks.stop()
        val = {}
        if validate:
            # tight reference at the last step's point: the plain method (CG, or MINRES for Hessians
            # that may be indefinite) to rtol 1e-7 from the computed w
            wref = w.clone()
            P.hessian_solve(wref, recycle=False, tol=1e-7, relative=True, maxit=6000, store_basis=False,
                            warm_start=True, allow_noconv=True, method=args.method)
            _, per_ref = P.hypergrad(wref, per_pair=True)
            err = (per - per_ref).norm(dim=1) / per_ref.norm(dim=1)
            mean_err = float((per.mean(0) - per_ref.mean(0)).norm() / per_ref.mean(0).norm())
            val["hg_err_max"] = float(err.max())
            val["hg_err_mean_grad"] = mean_err
        # per-kernel CUDA-event timing over further steps of the same sequence (profiling makes the
        # library launch the Krylov loop kernel by kernel, so every launch is bracketed by events)
        prof, ms_prof = None, None
        if prof_steps:
            P.profile(True)
            ev0.record(stream)
            for i in range(prof_steps):
                step(steps + i, False)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_prof = ev0.elapsed_time(ev1)
            prof = P.profile_read()
            P.profile(False)
        res = dict(ms=ms, iters=iters, prof=prof, ms_prof=ms_prof, launches=launches, clocks=ck,
                   graph_used=graph_used, **val)
        del P
        return res

    rec = run(strategy, args.steps, args.warmup, validate=True, profile_range=args.profile_range,
              prof_steps=args.prof_steps)
    cg = (run(parse("none"), args.steps, args.warmup, validate=True, prof_steps=args.prof_steps)
          if (args.compare_cg and strategy.recycles) else None)
    cold = (run(parse("none"), args.steps, args.warmup, validate=True, warm=False)
            if (args.compare_cg and args.cold and strategy.recycles) else None)
    e2e = run(strategy, args.steps, args.warmup, e2e=True) if args.e2e else None
    return dict(rec=rec, cg=cg, cold=cold, e2e=e2e, K=K, n_pix=n_pix, wl=wl, strategy=strategy, s_rec=s_rec, wdesc=wdesc)


# ---------------------------------------------------------------------------------------------
# CPU checker arm (bounded sample)

def oracle_sample(steps, warmup, max_seconds=None, strategy="RGen-L(R)", workload="batch64", variant="inner",
                  method="cg", rtol=0.0):
    """Run the FP64 checker on the smallest pair of the batch for warmup + steps outer steps, with
    the same refresh variant and Krylov method as the GPU arm.  Returns (seconds per timed step,
    sample description)."""
    from paper_2412_08264_gb300 import synth
    from paper_2412_08264_gb300.strategy import parse
    from oracle.bilevel import BilevelProblem, Adam
    from oracle.krylov import rcg, rminres
    from oracle.recycle import refresh, refresh_inner

    wl, s_rec, _ = make_workload(workload)
    k0 = min(range(len(wl.pairs)), key=lambda k: wl.pairs[k].height * wl.pairs[k].width)
    wl.pairs, wl.x_star, wl.noise, wl.masks = [wl.pairs[k0]], [wl.x_star[k0]], [wl.noise[k0]], [wl.masks[k0]]
    prob = BilevelProblem(wl)
    st = parse(strategy)
    ll = prob.lowers[0]
    theta = wl.theta0.copy()
    opt = Adam(ADAM_LR)
    x = np.zeros((ll.h, ll.w))
    w = np.zeros(ll.n)
    U = C = V = None
    AH_prev = None
    times = []
    g0 = np.linalg.norm(ll.grad(np.zeros_like(x), theta))
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        xs, _ = prob.solve_lower(theta, [x], gtol=LOWER_GTOL * g0)
        x = xs[0]
        AH = prob.apply_H(0, x, theta)
        if st.recycles and V is not None:
            Up = U if U is not None else np.zeros((ll.n, 0))
            Jfun = lambda v: prob.Jw(0, x, theta, v)   # noqa: E731
            if variant == "inner":
                U, C, Z, _ = refresh_inner(Up, V, AH_prev, AH, Jfun, s_rec, st.kind, st.size, st.side)
            else:
                U, C, Z, _ = refresh(Up, V, AH, Jfun, s_rec, st.kind, st.size, st.side)
        g = prob.rhs(0, x)
        tol = (rtol or workload_rtol(workload)) * np.linalg.norm(g)
        if method == "minres":
            out = rminres(AH, g, w, U, C, tol=tol, maxit=3000)
            out["V"] = out["V"][:, -MAX_BASIS:]
        else:
            out = rcg(AH, g, w, U, C, tol=tol, maxit=3000, kmax_store=None if variant == "inner" else MAX_BASIS)
        # inner: the first max_basis - 1 residuals (the Lanczos record); outer: the most recent max_basis
        w, V = out["w"], (out["V"][:, :MAX_BASIS - 1] if variant == "inner" else out["V"])
        AH_prev = AH
        hg = prob.Jw(0, x, theta, w)
        theta = opt.step(theta, hg)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
        if max_seconds is not None and sum(times) > max_seconds and len(times) >= 1:
            break
    desc = (f"pair {k0} of the {workload} batch ({ll.h}x{ll.w}, {wl.n_filters} {wl.filter_size}x{wl.filter_size} "
            f"filters), {strategy} ({variant} refresh, {'MINRES' if method == 'minres' else 'CG'}), "
            f"{warmup} warm-up + {len(times)} timed outer steps, FP64 NumPy")
    return float(np.mean(times)), len(times), desc


# ---------------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--strategy", default="RGen-L(R)")
    ap.add_argument("--workload", default="batch64", choices=["batch64", "inpaint", "deconv"],
                    help="batch64: the 64-pair deconvolution batch (the metric's workload); inpaint: 1024 "
                         "inpainting pairs shaped like the paper's Section 5.1 experiment; deconv: 512 "
                         "64x64 pairs shaped like its Section 5.2 experiment (use --method minres)")
    ap.add_argument("--refresh", default="inner", choices=["outer", "inner"],
                    help="recycle refresh: outer (eq. (3.3), current Hessian) or inner (eq. (3.4), the last "
                         "solve's Hessian through its Lanczos record; CG only)")
    ap.add_argument("--method", default="cg", choices=["cg", "minres"],
                    help="Krylov method of the Hessian solves: (recycled) CG or (recycled) MINRES")
    ap.add_argument("--max-basis", type=int, default=MAX_BASIS,
                    help="Krylov basis vectors kept per pair for the next refresh")
    ap.add_argument("--no-compare-cg", dest="compare_cg", action="store_false")
    ap.add_argument("--no-cold", dest="cold", action="store_false",
                    help="skip the cold-started plain solve (w_0 = 0 for every system)")
    ap.add_argument("--rtol", type=float, default=0.0,
                    help="residual stopping tolerance relative to ||g|| (default: the workload's)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--pairs", type=int, default=0, help="use only the first PAIRS pairs (profiling cases)")
    ap.add_argument("--prof-steps", type=int, default=2,
                    help="extra steps timed kernel by kernel with CUDA events (roofline, kernel_ms)")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="launch the Krylov and L-BFGS loops kernel by kernel from the host (profilers that "
                         "do not follow conditional CUDA-graph bodies see every launch)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.method == "minres":
        args.refresh = "outer"      # the Lanczos record of the inner refresh is kept by CG solves

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    metric = "hypergradients/s at 1e-4 rel. error (batched RCG vs plain CG); HVP HBM GB/s"

    if args.impl == "reference":
        if rank != 0:
            return
        sec, n, desc = oracle_sample(args.steps, args.warmup, strategy=args.strategy, workload=args.workload,
                                     variant=args.refresh, method=args.method, rtol=args.rtol)
        v = 1.0 / sec
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "hypergradients/s",
                          "n_gpus": args.gpus, "steps": n, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic",
                          "config": {"workload": {"batch64": "batch64_foe_n16f5", "inpaint": "inpaint1024x28_n3f5",
                                                  "deconv": "deconv512x64_n24f5"}[args.workload] + " (sample)",
                                     "strategy": args.strategy},
                          "cpu_baseline": {"value": v, "unit": "hypergradients/s", "cores": os.cpu_count(),
                                           "kind": "oracle", "sample": desc},
                          "e2e": {"value": v, "unit": "hypergradients/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    out = gpu_arm(args, rank, world, dist)
    rec, cg = out["rec"], out["cg"]
    K, n_pix, wl = out["K"], out["n_pix"], out["wl"]

    def tmax(ms):
        if world == 1:
            return ms
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms = tmax(rec["ms"])
    value = K * world * args.steps / (ms / 1e3)
    # roofline of the dominant kernel: the fused Hessian action of the Krylov loop
    zero = {"ms": 0.0, "launches": 0, "pixels": 0}
    profd = rec["prof"] or {k: zero for k in ["hvp", "hvp_multi", "grad", "jw", "krylov", "lbfgs", "gram", "gemm",
                                               "dense", "other"]}
    hv = profd["hvp"]
    masked = any(m is not None for m in wl.masks)
    fpp = hvp_flops_per_pixel(wl.n_filters, wl.filter_size, wl.pairs[0].blur_radius, masked)
    bpp = hvp_bytes_per_pixel(wl.n_filters, masked=masked)
    avg_ms = hv["ms"] / max(1, hv["launches"])
    flops_per_launch = fpp * hv["pixels"] / max(1, hv["launches"])
    ck = rec["clocks"] or {}
    peak_tflops = FP32_FMA_LANES * 2 * 2070e6 / 1e12
    if avg_ms > 0:
        achieved_tflops = flops_per_launch / (avg_ms / 1e3) / 1e12
        gbs = bpp * hv["pixels"] / max(1, hv["launches"]) / (avg_ms / 1e3) / 1e9
    else:   # no kernel-by-kernel pass (--prof-steps 0)
        achieved_tflops = gbs = None
    line = {
        "metric": metric, "value": value, "unit": "hypergradients/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": out["wdesc"] or (f"batch64_foe_n16f5: {K} pairs, sides 128-512, {n_pix} px, "
                                                f"16 5x5 filters, 9x9 blur, p={wl.n_params}"),
                   "strategy": out["strategy"].acronym(), "refresh": args.refresh, "krylov": args.method, "recycle_dim": out["s_rec"], "max_basis": args.max_basis,
                   "stop": f"residual rtol {args.rtol or workload_rtol(args.workload)}", "lower_gtol_rel": LOWER_GTOL, "outer": "Adam lr 1e-2",
                   "l2": "inputs larger than L2 (batch working set > 1 GB), no flush"},
        "hg_rel_err_max": rec.get("hg_err_max"), "hg_rel_err_mean_grad": rec.get("hg_err_mean_grad"),
        "krylov_iters_per_step": [int(np.max(it)) for it in rec["iters"]],
        "krylov_iters_total": int(np.sum(rec["iters"])),
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": None if achieved_tflops is None else achieved_tflops / peak_tflops,
                     "traffic": (HVP_DRAM_BYTES_PER_PIXEL * hv["pixels"] / max(1, hv["launches"])
                                 if (hv["launches"] and not masked) else None),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per pixel on the "
                                       "16-pair case, scaled to the launch's pixels",
                     "kernel": "k_foe_stencil<float,5,HVP> (fused blur + FoE Hessian action + dots)",
                     "flops_per_pixel": fpp, "pixels_per_launch": hv["pixels"] / max(1, hv["launches"]),
                     "avg_launch_ms": avg_ms, "hbm_gbs_algorithmic": gbs,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "share_of_step": hv["ms"] / max(1e-9, rec["ms_prof"] or 1e-9),
                     "timing": f"CUDA events around every launch over {args.prof_steps} further steps "
                               "(stream path)"},
        "kernel_ms": {k: round(v["ms"], 3) for k, v in profd.items()},
        "kernel_ms_steps": args.prof_steps, "profiled_ms_per_step": (rec["ms_prof"] or 0) / max(1, args.prof_steps),
        "krylov_graph": rec["graph_used"],
        "gpu_launches": rec["launches"],
        "clocks": ck,
    }
    if cg is not None:
        ms_cg = tmax(cg["ms"])
        line["plain_cg"] = {"value": K * world * args.steps / (ms_cg / 1e3), "ms_per_step": ms_cg / args.steps,
                            "krylov_iters_total": int(np.sum(cg["iters"])), "hg_rel_err_max": cg.get("hg_err_max"),
                            "kernel_ms": ({k: round(v["ms"], 3) for k, v in cg["prof"].items()} if cg["prof"] else None),
                            "hvp_avg_launch_ms": (cg["prof"]["hvp"]["ms"] / max(1, cg["prof"]["hvp"]["launches"])
                                                  if cg["prof"] else None)}
    if out["cold"] is not None:
        cold = out["cold"]
        ms_c = tmax(cold["ms"])
        line["plain_cg_cold"] = {"value": K * world * args.steps / (ms_c / 1e3), "ms_per_step": ms_c / args.steps,
                                 "krylov_iters_total": int(np.sum(cold["iters"])),
                                 "hg_rel_err_max": cold.get("hg_err_max")}
    if out["e2e"] is not None:
        ms_e = tmax(out["e2e"]["ms"])
        h2d = 2 * n_pix * 4 + wl.n_params * 8
        line["e2e"] = {"value": K * world * args.steps / (ms_e / 1e3), "unit": "hypergradients/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": wl.n_params * 8}
    if rank == 0 and world == 1 and args.cpu_baseline:
        sec, n, desc = oracle_sample(2, 1, max_seconds=30.0, strategy=args.strategy, workload=args.workload,
                                     variant=args.refresh, method=args.method, rtol=args.rtol)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "hypergradients/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
