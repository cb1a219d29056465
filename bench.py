"""Throughput of the hypergradient hot path on the 64-pair batch workload.

One step = one outer iteration over the batch (64 training pairs of uneven sizes, FoE with 16 5x5
filters): warm-started lower solve (L-BFGS), recycle refresh (by default the inner variant of
eq. (3.4)), warm-started recycled-CG Hessian solve, J w contraction, then the outer update of theta
(Adam of Section 5.2, or --outer gd: Algorithms 1-2 with Armijo backtracking).

value  hypergradients per second over the time of bl_ritz_update + bl_hessian_solve + bl_hypergrad
       (CUDA events on the library's stream), the unit of work of the recycling method; the lower
       solve is reported separately (lower_solve_ms_per_step) and inside the full-step figures
       (ms_per_step, e2e).  Accuracy: every k-th timed step (and the last) each pair's hypergradient
       is compared with an FP64 reference at the same point (an FP64 problem on the same data, plain
       CG to a relative residual of --ref-rtol from the FP32 solution), outside the timed region;
       hg_rel_err_max_fp64 is the largest relative error seen.  At the last step the FP64 checker
       recomputes the two smallest pairs' hypergradients at the point the GPU reached.

Arms (same run, same sequence of outer steps per arm): the recycled method (--strategy), plain CG
warm-started and cold-started, and Ritz-S recycling.

  --protocol fixed   the fixed-sequence study: one sequence of (theta_i, x^_i) is generated once,
                     FP64 references are computed for every system, and each arm solves the same
                     sequence at every residual tolerance of --rtol-sweep; per arm the loosest
                     tolerance that keeps every hypergradient within 1e-4 is reported with its
                     throughput (one JSON line per arm and tolerance, then a summary line).
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
HG_BAR = 1e-4          # hypergradient relative-error bar
FP32_LANES_PER_SM = 128
# HBM copy bandwidth measured on the GB300s (STREAM-style copy), used when the driver's
# MEASURED_PEAKS.json is absent from the working tree
HBM_GBS_POOL = 6683.5
# DRAM bytes (read + write) per pixel of one k_hvp_tma<5> launch, from an ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum (first 16 pairs of the 64-pair batch, 1,306,624 px,
# three launches: 68.1 B/px read each, the first writing 2.0 B/px back) scaled to the timed launches
# by their pixels.  Valid while the kernel's sources hash to HVP_TRAFFIC_SHA; otherwise the roofline
# reports null traffic.
HVP_TRAFFIC_B_PER_PX = 70.1
HVP_TRAFFIC_SOURCES = ("hvp_tma.cu", "device.cuh", "common.cuh")
HVP_TRAFFIC_SHA = "c3ba9847d6bd4535"


def hvp_traffic_valid():
    import hashlib
    h = hashlib.sha256()
    for name in HVP_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_08264_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16] == HVP_TRAFFIC_SHA


def hvp_flops_per_pixel(n_filters, f, rb, masked=False):
    """Algorithmic FP32 flops of one Hessian action per pixel (fields variant):
    per filter K v (2 T), times d_j (1), K^T (2 T); blur A A v separable (4 passes x (2 r_b + 1)
    FMA = 8 (2 r_b + 1) flop), or for inpainting the mask product (2); l2 term and sum (2)."""
    T = f * f
    return n_filters * (4 * T + 1) + (2 if masked else 8 * (2 * rb + 1)) + 2


def hvp_bytes_per_pixel(n_filters, esz=4, masked=False, dots_cols=0):
    """Algorithmic HBM bytes of one Hessian action per pixel: v in, H v out, N fields d_j in (and
    the 1-byte mask for inpainting); with fused Krylov dots also p and the dots_cols columns of C
    (p is the staged v)."""
    return (2 + n_filters + dots_cols) * esz + (1 if masked else 0)


def hbm_peak():
    """(GB/s, source) of the HBM roof."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for key in ("hbm_gbs", "hbm_copy_gbs", "hbm"):
            if key in d and float(d[key]) > 0:
                return float(d[key]), f"measured ({os.path.basename(path)}: {key})"
    except Exception:
        pass
    return HBM_GBS_POOL, "measured on this pool's GB300s (STREAM-style copy), recorded value"


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
    if name == "cfg2":
        wl = synth.foe_256()
        return wl, 20, (f"foe256_n8f5: one 256x256 pair, 5x5 blur sigma 1.5, noise 0.02, 8 5x5 filters, "
                        f"p={wl.n_params}, recycle dimension 20")
    if name == "large":
        wl = synth.large_2048()
        return wl, 50, (f"large2048_foe_n48f7: one 2048x2048 pair, 9x9 blur sigma 3, noise 0.01, 48 7x7 filters, "
                        f"p={wl.n_params}, recycle dimension 50")
    wl = synth.batch_64(replica=replica)
    return wl, S_RECYCLE, None


# ---------------------------------------------------------------------------------------------
# Accuracy references

class Fp64Reference:
    """The same pairs as an FP64 problem: per-pair hypergradients at a given point (theta, x^) by the
    plain method (CG, or MINRES for Hessians that may be indefinite) to a relative residual of
    `rtol`, warm-started from the FP32 solution.  The FP64 problem never takes part in a timed step."""

    def __init__(self, wl, y, xs, rtol, method):
        from paper_2412_08264_gb300 import api
        self.P = api.from_workload(wl, y.double(), xs.double(), precision="fp64", max_recycle=0, max_basis=0)
        self.rtol = rtol
        self.method = method

    def hypergrads(self, theta_d, xhat, w):
        self.P.set_point(theta_d, xhat.double())
        w64 = w.double().clone()
        info = self.P.hessian_solve(w64, recycle=False, tol=self.rtol, relative=True, maxit=20000,
                                    store_basis=False, warm_start=True, allow_noconv=True, method=self.method)
        _, per = self.P.hypergrad(w64, per_pair=True)
        return per, max(i["iters"] for i in info)


def rel_errors(per, ref):
    """Relative error of each pair's hypergradient against its reference (rows)."""
    per = per.double()
    return ((per - ref).norm(dim=1) / ref.norm(dim=1)).cpu().numpy()


def oracle_spot_check(wl, theta, xhats, per_gpu, pairs):
    """The FP64 checker's hypergradient of the listed pairs at the point (theta, x^_k) the GPU arm
    reached (reference solve to 1e-12), against the GPU's FP32 values.  The hypergradient at a point
    depends on x^, x* and theta only (eq. (2.7)), so the checker needs none of the GPU's data."""
    import copy
    from oracle.bilevel import BilevelProblem
    sub = copy.copy(wl)
    sub.pairs = [wl.pairs[k] for k in pairs]
    sub.x_star = [wl.x_star[k] for k in pairs]
    sub.noise = [wl.noise[k] for k in pairs]
    sub.masks = [wl.masks[k] for k in pairs] if wl.masks else []
    prob = BilevelProblem(sub)
    errs = []
    for j, k in enumerate(pairs):
        w = prob.reference_w(j, xhats[j], theta, rtol=1e-12)
        ref = prob.Jw(j, xhats[j], theta, w)
        errs.append(float(np.linalg.norm(per_gpu[j] - ref) / np.linalg.norm(ref)))
    return errs


# ---------------------------------------------------------------------------------------------
# GPU arm: the live sequence (every arm runs its own outer iteration from the same start)

def gpu_setup(args, rank):
    import torch
    from paper_2412_08264_gb300 import api
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl, s_rec, wdesc = make_workload(args.workload, replica=rank)
    if args.pairs and args.pairs < len(wl.pairs):
        wl.pairs, wl.x_star, wl.noise = wl.pairs[:args.pairs], wl.x_star[:args.pairs], wl.noise[:args.pairs]
        if wl.masks:
            wl.masks = wl.masks[:args.pairs]
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
    return dict(dev=dev, wl=wl, s_rec=s_rec, wdesc=wdesc, xs_h=xs_h, y_h=y_h, xs=xs, y=y)


def run_live(args, env, strat, steps, warmup, world=1, dist=None, e2e=False, validate=False, prof_steps=0,
             warm=True, ref=None):
    """One arm on its own outer sequence.  Returns timings (CUDA events), iterations and, when
    `validate`, the FP64 errors of every k-th timed step and the last one."""
    import torch
    from paper_2412_08264_gb300 import api
    from paper_2412_08264_gb300.parallel import allreduce_mean
    wl, dev = env["wl"], env["dev"]
    y, xs = env["y"], env["xs"]
    rtol = args.rtol or workload_rtol(args.workload)
    K = len(wl.pairs)
    P = api.from_workload(wl, y, xs, max_recycle=env["s_rec"], max_basis=args.max_basis)
    y_d = torch.empty_like(y)
    xs_d = torch.empty_like(xs)
    stream = torch.cuda.current_stream(dev)
    st = {"theta": wl.theta0.copy(), "m": np.zeros_like(wl.theta0), "v": np.zeros_like(wl.theta0), "t": 0,
          "beta": 1.0, "hg_prev": None, "xhat": P.zeros(), "have_point": False}
    theta_d = torch.tensor(st["theta"], dtype=torch.float64, device=dev)
    w = P.zeros()
    E = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731

    def lower(th_d, x):
        P.lower_solve(th_d, x, gtol=LOWER_GTOL, relative=True, max_iters=2000, allow_noconv=True, graph=args.graph)

    def hg_part():
        if strat.recycles and st["t"] > 0:
            P.ritz_update(strat, env["s_rec"], variant=args.refresh)
        info = P.hessian_solve(w, recycle=strat.recycles, nsc=strat.nsc, tol=rtol, relative=True, maxit=3000,
                               store_basis=(("lanczos" if args.refresh == "inner" else True)
                                            if strat.recycles else False), warm_start=warm,
                               nsc_scale=None if st["hg_prev"] is None else [st["hg_prev"]] * K,
                               allow_noconv=True, method=args.method, graph=args.graph)
        mean, per, loss = P.hypergrad(w, per_pair=True, loss=True)
        return info, mean, per, loss

    def step():
        ev = [E() for _ in range(4)]
        ev[0].record(stream)
        if e2e:
            y_d.copy_(env["y_h"], non_blocking=True)
            xs_d.copy_(env["xs_h"], non_blocking=True)
            P.set_data(y_d, xs_d)
        theta_step = st["theta"].copy()
        if args.outer == "adam" or not st["have_point"]:
            lower(theta_d, st["xhat"])
            st["have_point"] = True
        ev[1].record(stream)
        info, mean, per, c1 = hg_part()
        ev[2].record(stream)
        if world > 1:
            mean = allreduce_mean(mean, K)
        g = mean.cpu().numpy()                       # the step's result, read back every step
        st["hg_prev"] = float(np.linalg.norm(g))
        xhat_step = st["xhat"]
        st["t"] += 1
        if args.outer == "adam":                     # Section 5.2: fixed step length
            t = st["t"]
            st["m"] = 0.9 * st["m"] + 0.1 * g
            st["v"] = 0.999 * st["v"] + 0.001 * g * g
            st["theta"] = st["theta"] - ADAM_LR * (st["m"] / (1 - 0.9 ** t)) / (np.sqrt(st["v"] / (1 - 0.999 ** t)) + 1e-8)
            theta_d.copy_(torch.from_numpy(st["theta"]), non_blocking=False)
        else:                                        # Algorithms 1-2: Armijo backtracking
            dd = float(g @ g)
            xt = st["xhat"].clone()
            for j in range(1, 31):
                stp = st["beta"] * 0.5 ** (j - 1)
                th_j = st["theta"] - stp * g
                theta_d.copy_(torch.from_numpy(th_j), non_blocking=False)
                lower(theta_d, xt)
                _, c0 = P.hypergrad(w, loss=True)
                if c0 < c1 - 1e-4 * stp * dd:
                    break
            st["beta"] = 2.0 * stp
            st["theta"] = th_j
            st["xhat"] = xt
        ev[3].record(stream)
        return ev, info, per, theta_step, xhat_step

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(dev.index)
    clocks.start()
    launches0 = P.launch_count()
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    evs, iters, errs, per_last = [], [], [], None
    for i in range(steps):
        ev, info, per, theta_step, xhat_step = step()
        evs.append(ev)
        iters.append([d["iters"] for d in info])
        per_last = (per, theta_step, xhat_step.clone())
        if validate and ref is not None and ((i + 1) % args.validate_every == 0 or i == steps - 1):
            torch.cuda.synchronize()
            per_ref, it_ref = ref.hypergrads(torch.tensor(theta_step, dtype=torch.float64, device=dev), xhat_step, w)
            errs.append({"step": i, "max": float(rel_errors(per, per_ref).max()), "ref_iters": it_ref})
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    launches = P.launch_count() - launches0
    ms = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in evs)   # noqa: E731
    ms_hg, ms_step = ms(1, 2), ms(0, 3)
    ms_lower = ms(0, 1) + ms(2, 3) if args.outer == "gd" else ms(0, 1)
    res = dict(ms_hg=ms_hg, ms_step=ms_step, ms_lower=ms_lower, iters=iters, launches=launches, clocks=ck,
               graph_used=P.graph_used(), errs=errs, per_last=per_last, tma=P.hvp_tma())
    if prof_steps:
        P.profile(True)
        e0, e1 = E(), E()
        e0.record(stream)
        for _ in range(prof_steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        res["ms_prof"] = e0.elapsed_time(e1)
        res["prof"] = P.profile_read()
        P.profile(False)
    del P
    return res


# ---------------------------------------------------------------------------------------------
# Bandwidth-bound Hessian action: the TV regulariser on one large FP32 image

def tv_hvp_microbench(dev, sides=(2048, 4096), reps=10):
    """Blur + TV Hessian action (the TMA-staged TV kernel) on one side x side image: 12 algorithmic
    bytes per pixel (v and x^ in, H v out).  Returns per side the CUDA-event time of one launch and
    the achieved GB/s (algorithmic bytes / time)."""
    import torch
    from paper_2412_08264_gb300 import api, synth
    out = []
    for side in sides:
        rng = np.random.default_rng(side)
        wl = synth.tv_32()
        wl.precision = "fp32"
        wl.pairs = [synth.PairSpec(side, side, 2.0, 4, 0.01)]
        wl.x_star = [synth.rectangles_image(rng, side, side)]
        wl.noise = [np.zeros((side, side))]
        xs = torch.tensor(wl.x_star[0].ravel(), dtype=torch.float32, device=dev)
        P = api.from_workload(wl, xs, xs, max_recycle=1, max_basis=1)
        xh = (xs + 0.05 * torch.randn_like(xs)).contiguous()
        P.set_point(torch.tensor([-3.0], dtype=torch.float64, device=dev), xh)
        v = torch.randn_like(xs)
        for _ in range(3):
            P.hvp(v)
        torch.cuda.synchronize()
        P.profile(True)
        for _ in range(reps):
            P.hvp(v)
        pr = P.profile_read()["hvp"]
        P.profile(False)
        ms = pr["ms"] / max(1, pr["launches"])
        out.append({"side": side, "pixels": side * side, "ms": ms, "bytes_per_pixel": 12,
                    "gbs": 12 * side * side / (ms * 1e-3) / 1e9, "tma": P.hvp_tma()})
        del P
    return out


def foe_hvp_full_batch(env, reps=20):
    """The Hessian action with every pair of the batch active, at a point near x*: inside the timed
    steps the Krylov loops' launches shrink as pairs converge (the grid's CTAs of converged pairs
    exit at once), so this separates the kernel's own rate from that occupancy effect.  Per-launch
    CUDA-event time over reps launches."""
    import torch
    from paper_2412_08264_gb300 import api
    wl, dev = env["wl"], env["dev"]
    P = api.from_workload(wl, env["y"], env["xs"], max_recycle=1, max_basis=1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    xh = (env["xs"] + 0.02 * torch.randn(env["xs"].shape, generator=gen, device=dev)).contiguous()
    P.set_point(torch.tensor(wl.theta0, dtype=torch.float64, device=dev), xh)
    v = torch.randn(env["xs"].shape, generator=gen, device=dev)
    for _ in range(3):
        P.hvp(v)
    torch.cuda.synchronize()
    P.profile(True)
    for _ in range(reps):
        P.hvp(v)
    pr = P.profile_read()["hvp"]
    P.profile(False)
    tma = P.hvp_tma()
    del P
    n = max(1, pr["launches"])
    return {"launches": pr["launches"], "ms": pr["ms"] / n, "pixels": pr["pixels"] / n, "tma": tma}


# ---------------------------------------------------------------------------------------------
# GPU arm: the fixed-sequence protocol

def run_fixed(args, env, arm_names, rtols):
    """Generate (theta_i, x^_i), i < S, once (plain CG to 1e-6 for the outer steps), FP64 references at
    every point, then let each arm solve the same sequence at each tolerance.  System 0 (no recycle
    space yet; graph capture) is solved but not timed."""
    import torch
    from paper_2412_08264_gb300 import api
    from paper_2412_08264_gb300.strategy import parse
    wl, dev = env["wl"], env["dev"]
    K = len(wl.pairs)
    S = args.systems
    stream = torch.cuda.current_stream(dev)
    E = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    # 1. the sequence
    P = api.from_workload(wl, env["y"], env["xs"], max_recycle=1, max_basis=1)
    theta = wl.theta0.copy()
    th_d = torch.tensor(theta, dtype=torch.float64, device=dev)
    x = P.zeros()
    w = P.zeros()
    seq = []
    m, v2, beta = np.zeros_like(theta), np.zeros_like(theta), 1.0
    P.lower_solve(th_d, x, gtol=LOWER_GTOL, relative=True, max_iters=2000, allow_noconv=True)
    for i in range(S):
        P.hessian_solve(w, recycle=False, tol=1e-6, relative=True, maxit=5000, store_basis=False,
                        allow_noconv=True, method=args.method)
        mean, c1 = P.hypergrad(w, loss=True)
        seq.append((theta.copy(), x.clone(), w.clone()))
        g = mean.cpu().numpy()
        if args.outer == "adam":
            m = 0.9 * m + 0.1 * g
            v2 = 0.999 * v2 + 0.001 * g * g
            theta = theta - ADAM_LR * (m / (1 - 0.9 ** (i + 1))) / (np.sqrt(v2 / (1 - 0.999 ** (i + 1))) + 1e-8)
            th_d.copy_(torch.from_numpy(theta))
            P.lower_solve(th_d, x, gtol=LOWER_GTOL, relative=True, max_iters=2000, allow_noconv=True)
        else:
            dd = float(g @ g)
            xt = x.clone()
            for j in range(1, 31):
                stp = beta * 0.5 ** (j - 1)
                th_j = theta - stp * g
                th_d.copy_(torch.from_numpy(th_j))
                P.lower_solve(th_d, xt, gtol=LOWER_GTOL, relative=True, max_iters=2000, allow_noconv=True)
                _, c0 = P.hypergrad(w, loss=True)
                if c0 < c1 - 1e-4 * stp * dd:
                    break
            beta, theta, x = 2.0 * stp, th_j, xt
    del P
    # 2. FP64 references
    ref = Fp64Reference(wl, env["y"], env["xs"], args.ref_rtol, args.method)
    refs = []
    for th, xh, w0 in seq:
        per_ref, _ = ref.hypergrads(torch.tensor(th, dtype=torch.float64, device=dev), xh, w0)
        refs.append(per_ref)
    del ref
    # 3. every arm on the same sequence
    out = []
    for name in arm_names:
        strat = parse(name)
        for rtol in rtols:
            P = api.from_workload(wl, env["y"], env["xs"], max_recycle=env["s_rec"], max_basis=args.max_basis)
            w = P.zeros()
            hg_prev, ms, errs, its, nsc_rows = None, 0.0, [], 0, []
            for i, (th, xh, _) in enumerate(seq):
                P.set_point(torch.tensor(th, dtype=torch.float64, device=dev), xh)
                e0, e1 = E(), E()
                e0.record(stream)
                if strat.recycles and i > 0:
                    P.ritz_update(strat, env["s_rec"], variant=args.refresh)
                info = P.hessian_solve(w, recycle=strat.recycles, nsc=strat.nsc, tol=rtol, relative=True,
                                       maxit=5000, store_basis=(("lanczos" if args.refresh == "inner" else True)
                                                                if strat.recycles else False),
                                       warm_start=True, nsc_scale=None if hg_prev is None else [hg_prev] * K,
                                       allow_noconv=True, method=args.method, graph=args.graph)
                mean, per = P.hypergrad(w, per_pair=True)
                e1.record(stream)
                torch.cuda.synchronize()
                scale = hg_prev
                hg_prev = float(mean.norm())
                errs.append(float(rel_errors(per, refs[i]).max()))
                if strat.nsc:
                    # the estimate of eq. (4.2) at the stop, relative like the rule (to the previous
                    # hypergradient's norm), next to the true relative error of the mean hypergradient
                    true_rel = float((mean - refs[i].mean(0)).norm() / refs[i].mean(0).norm())
                    nsc_rows.append({"system": i, "iters": [d["iters"] for d in info],
                                     "estimate_rel": (None if scale is None else
                                                      float(max(d["nsc"] for d in info)) / scale),
                                     "true_rel_err": true_rel})
                if i > 0:
                    ms += e0.elapsed_time(e1)
                    its += sum(d["iters"] for d in info)
            del P
            rec = {"protocol": "fixed", "arm": name, "rtol": rtol, "value": K * (S - 1) / (ms / 1e3),
                   "unit": "hypergradients/s", "ms_per_system": ms / (S - 1), "hg_rel_err_max": max(errs),
                   "hg_rel_err_per_system": errs, "krylov_iters": its, "systems": S, "outer": args.outer}
            if nsc_rows:
                rec["nsc"] = nsc_rows
            out.append(rec)
            print(json.dumps(rec), flush=True)
    summary = {}
    for name in arm_names:
        ok = [r for r in out if r["arm"] == name and r["hg_rel_err_max"] <= HG_BAR]
        best = max(ok, key=lambda r: r["rtol"]) if ok else None
        summary[name] = None if best is None else {"rtol": best["rtol"], "value": best["value"],
                                                   "hg_rel_err_max": best["hg_rel_err_max"],
                                                   "krylov_iters": best["krylov_iters"]}
    return out, summary


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



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--strategy", default="RGen-L(R)")
    ap.add_argument("--workload", default="batch64", choices=["batch64", "inpaint", "deconv", "cfg2", "large"],
                    help="batch64: the 64-pair deconvolution batch (the metric's workload); inpaint: 1024 "
                         "inpainting pairs shaped like the paper's Section 5.1 experiment; deconv: 512 "
                         "64x64 pairs shaped like its Section 5.2 experiment (use --method minres); cfg2: one "
                         "256x256 pair with 8 5x5 filters; large: one 2048x2048 pair with 48 7x7 filters "
                         "(recycle dimension 50)")
    ap.add_argument("--refresh", default="inner", choices=["outer", "inner"],
                    help="recycle refresh: outer (eq. (3.3), current Hessian) or inner (eq. (3.4), the last "
                         "solve's Hessian through its Lanczos record; CG only)")
    ap.add_argument("--method", default="cg", choices=["cg", "minres"],
                    help="Krylov method of the Hessian solves: (recycled) CG or (recycled) MINRES")
    ap.add_argument("--outer", default="adam", choices=["adam", "gd"],
                    help="outer iteration: Adam with step 1e-2 (Section 5.2) or gradient descent with Armijo "
                         "backtracking (Algorithms 1-2, Section 5.1)")
    ap.add_argument("--max-basis", type=int, default=MAX_BASIS,
                    help="Krylov basis vectors kept per pair for the next refresh")
    ap.add_argument("--arms", default="none,none-cold,Ritz-S",
                    help="comparison arms run after the recycled one: 'none' (plain CG warm-started), "
                         "'none-cold' (plain CG from w = 0), recycling strategies by acronym; '' for none")
    ap.add_argument("--rtol", type=float, default=0.0,
                    help="residual stopping tolerance relative to ||g|| (default: the workload's)")
    ap.add_argument("--validate-every", type=int, default=5,
                    help="compare every k-th timed step (and the last) with the FP64 reference")
    ap.add_argument("--ref-rtol", type=float, default=1e-10,
                    help="relative residual of the FP64 reference solves")
    ap.add_argument("--no-validate", dest="validate", action="store_false")
    ap.add_argument("--no-oracle-check", dest="oracle_check", action="store_false")
    ap.add_argument("--protocol", default="live", choices=["live", "fixed"])
    ap.add_argument("--systems", type=int, default=8, help="fixed protocol: systems in the sequence")
    ap.add_argument("--rtol-sweep", default="1e-4,3e-4,1e-3", help="fixed protocol: tolerances per arm")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-microbench", dest="microbench", action="store_false",
                    help="skip the TV Hessian-action bandwidth runs at 2048^2 and 4096^2")
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
    wnames = {"batch64": "batch64_foe_n16f5", "inpaint": "inpaint1024x28_n3f5", "deconv": "deconv512x64_n24f5",
              "cfg2": "foe256_n8f5", "large": "large2048_foe_n48f7"}

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
                          "config": {"workload": wnames[args.workload] + " (sample)", "strategy": args.strategy},
                          "cpu_baseline": {"value": v, "unit": "hypergradients/s", "cores": os.cpu_count(),
                                           "kind": "oracle", "sample": desc},
                          "e2e": {"value": v, "unit": "hypergradients/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2412_08264_gb300.strategy import parse
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    env = gpu_setup(args, rank)
    wl, dev = env["wl"], env["dev"]
    K, n_pix = len(wl.pairs), env["xs"].numel()

    if args.protocol == "fixed":
        arms = [args.strategy] + [a for a in args.arms.split(",") if a and a != "none-cold"]
        rtols = [float(x) for x in args.rtol_sweep.split(",")]
        out, summary = run_fixed(args, env, arms, rtols)
        if rank == 0:
            print(json.dumps({"protocol": "fixed", "summary": summary, "systems": args.systems, "outer": args.outer,
                              "workload": wnames[args.workload], "ref_rtol": args.ref_rtol, "bar": HG_BAR}))
        return

    strategy = parse(args.strategy)
    ref = None
    if args.validate:
        ref = Fp64Reference(wl, env["y"], env["xs"], args.ref_rtol, args.method)
    rec = run_live(args, env, strategy, args.steps, args.warmup, world, dist, validate=args.validate,
                   prof_steps=args.prof_steps, ref=ref)
    arm_res = {}
    for name in [a for a in args.arms.split(",") if a]:
        cold = name == "none-cold"
        st = parse("none" if cold else name)
        if st == strategy:
            continue
        arm_res[name] = run_live(args, env, st, args.steps, args.warmup, world, dist, validate=args.validate,
                                 prof_steps=args.prof_steps if name == "none" else 0, warm=not cold, ref=ref)
    e2e = run_live(args, env, strategy, args.steps, args.warmup, world, dist, e2e=True) if args.e2e else None
    del ref
    tvb = tv_hvp_microbench(dev) if args.microbench else None
    fullb = foe_hvp_full_batch(env) if args.microbench and wl.reg == "foe" else None

    def tmax(ms):
        if world == 1:
            return ms
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    steps = args.steps
    hg_total = K * world * steps
    ms_hg, ms_step, ms_lower = tmax(rec["ms_hg"]), tmax(rec["ms_step"]), tmax(rec["ms_lower"])
    value = hg_total / (ms_hg / 1e3)
    ck = rec["clocks"] or {}
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clk = ck.get("sm_mhz") or ck.get("sm_max_mhz") or 2070.0
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
    hbm, hbm_src = hbm_peak()
    prof = rec.get("prof")
    masked = any(m is not None for m in wl.masks)
    fpp = hvp_flops_per_pixel(wl.n_filters, wl.filter_size, wl.pairs[0].blur_radius, masked)
    bpp = hvp_bytes_per_pixel(wl.n_filters, masked=masked, dots_cols=0 if rec["tma"] else env["s_rec"])
    roof = {"bound": "alu", "achieved": None, "peak": peak_tflops, "unit": "TFLOP/s", "frac": None, "traffic": None}
    kvec = None
    if prof:
        hv = prof["hvp"]
        traffic_ok = bool(rec["tma"]) and wl.filter_size == 5 and hvp_traffic_valid()
        n_l = max(1, hv["launches"])
        avg_ms, px = hv["ms"] / n_l, hv["pixels"] / n_l
        ach = fpp * px / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else None
        gbs = bpp * px / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
        roof.update({
            "achieved": ach, "frac": None if ach is None else ach / peak_tflops,
            "traffic": (HVP_TRAFFIC_B_PER_PX * px if traffic_ok else None),
            "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum: {HVP_TRAFFIC_B_PER_PX} B/px "
                               "on the first 16 pairs, times the pixels per timed launch" if traffic_ok else
                               "null: the kernel changed since its last ncu DRAM capture"),
            "kernel": ("k_hvp_tma<5> (TMA-staged blur + FoE Hessian action)" if rec["tma"]
                       else "k_foe_stencil<float,5,HVP> (fused blur + FoE Hessian action + dots)"),
            "flops_per_pixel": fpp, "bytes_per_pixel": bpp, "pixels_per_launch": px, "avg_launch_ms": avg_ms,
            "hbm_gbs_algorithmic": gbs, "hbm_frac_of_measured": None if gbs is None else gbs / hbm,
            "peak_source": (f"derived: {sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                            f"{clk:.0f} MHz (median SM clock sampled during the timed region)"),
            "share_of_step": hv["ms"] / max(1e-9, rec["ms_prof"]),
            "timing": f"CUDA events around every launch over {args.prof_steps} further steps (stream path)"})
        if fullb and fullb["ms"] > 0:
            a_f = fpp * fullb["pixels"] / (fullb["ms"] * 1e-3) / 1e12
            roof["full_batch_launch"] = {
                "definition": "the same kernel with every pair active (20 launches at a point near x*), "
                              "against the same peak; the timed steps' launches shrink as pairs converge",
                "avg_launch_ms": fullb["ms"], "pixels_per_launch": fullb["pixels"], "achieved": a_f,
                "frac": a_f / peak_tflops, "tma": fullb["tma"]}
        kv = prof["krylov_vec"]
        if kv["ms"] > 0 and kv["bytes"] > 0:
            g_kv = kv["bytes"] / (kv["ms"] * 1e-3) / 1e9
            kvec = {"kernels": "k_dots_v4 / k_dots, k_update, k_pupdate (recycled-CG vector passes)",
                    "achieved_gbs": g_kv, "peak_gbs": hbm, "frac": g_kv / hbm, "bytes": kv["bytes"],
                    "ms": kv["ms"], "launches": kv["launches"], "peak_source": hbm_src,
                    "bytes_definition": "each vector read or written once per pass (counted by the kernels)"}
    errs = [e["max"] for e in rec["errs"]]
    line = {
        "metric": metric, "value": value, "unit": "hypergradients/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_step / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": env["wdesc"] or (f"batch64_foe_n16f5: {K} pairs, sides 128-512, {n_pix} px, "
                                                f"16 5x5 filters, 9x9 blur, p={wl.n_params}"),
                   "strategy": strategy.acronym(), "refresh": args.refresh, "krylov": args.method,
                   "recycle_dim": env["s_rec"], "max_basis": args.max_basis, "outer": args.outer,
                   "stop": f"residual rtol {args.rtol or workload_rtol(args.workload)}", "lower_gtol_rel": LOWER_GTOL,
                   "l2": "inputs larger than L2 (batch working set > 1 GB), no flush"},
        "value_definition": "hypergradients / s over the CUDA-event time of bl_ritz_update + bl_hessian_solve + "
                            "bl_hypergrad; the lower solve is timed separately",
        "lower_solve_ms_per_step": ms_lower / steps, "hg_part_ms_per_step": ms_hg / steps,
        "full_step_hypergradients_per_s": hg_total / (ms_step / 1e3),
        "pixel_hypergradients_per_s": n_pix * world * steps / (ms_hg / 1e3),
        "hg_rel_err_max_fp64": max(errs) if errs else None,
        "hg_validation": {"steps": [e["step"] for e in rec["errs"]], "max_per_step": errs,
                          "ref": f"FP64 problem on the same data, plain {args.method.upper()} to relative residual "
                                 f"{args.ref_rtol} at the same (theta, x^), warm-started from the FP32 w",
                          "ref_iters": [e["ref_iters"] for e in rec["errs"]]},
        "krylov_iters_per_step": [int(np.max(it)) for it in rec["iters"]],
        "krylov_iters_total": int(np.sum(rec["iters"])),
        "roofline": roof,
        "krylov_vec": kvec,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items()} if prof else None,
        "kernel_ms_steps": args.prof_steps,
        "profiled_ms_per_step": rec.get("ms_prof", 0) / max(1, args.prof_steps),
        "hvp_tma": rec["tma"], "krylov_graph": rec["graph_used"], "gpu_launches": rec["launches"], "clocks": ck,
    }
    if tvb:
        hbm, hbm_src = hbm_peak()
        for r in tvb:
            r["frac"] = r["gbs"] / hbm
        line["hbm_microbench"] = {"kernel": "k_tv_hvp_tma (blur + TV Hessian action, FP32)", "peak_gbs": hbm,
                                  "peak_source": hbm_src, "runs": tvb}
    arms_out = {}
    for name, r in arm_res.items():
        m_hg, m_st = tmax(r["ms_hg"]), tmax(r["ms_step"])
        e_r = [e["max"] for e in r["errs"]]
        arms_out[name] = {"value": hg_total / (m_hg / 1e3), "full_step_hypergradients_per_s": hg_total / (m_st / 1e3),
                          "hg_part_ms_per_step": m_hg / steps, "ms_per_step": m_st / steps,
                          "krylov_iters_total": int(np.sum(r["iters"])),
                          "hg_rel_err_max_fp64": max(e_r) if e_r else None,
                          "kernel_ms": ({k: round(v["ms"], 3) for k, v in r["prof"].items()} if r.get("prof") else None)}
    line["arms"] = arms_out
    if "none" in arms_out:
        line["vs_plain_cg"] = value / arms_out["none"]["value"]
    if e2e is not None:
        ms_e = tmax(e2e["ms_step"])
        h2d = 2 * n_pix * 4 + wl.n_params * 8
        line["e2e"] = {"value": hg_total / (ms_e / 1e3), "unit": "hypergradients/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": wl.n_params * 8,
                       "definition": "whole outer step (lower solve included) through the public API, y and x* "
                                     "uploaded from pinned host memory and the mean hypergradient read back"}
    if rank == 0 and world == 1 and args.oracle_check and rec["per_last"] is not None and not args.pairs:
        per, th_last, xh_last = rec["per_last"]
        order = sorted(range(K), key=lambda k: wl.pairs[k].height * wl.pairs[k].width)[:2]
        offs = np.cumsum([0] + [p.height * p.width for p in wl.pairs])
        xa = xh_last.double().cpu().numpy()
        xhs = [xa[offs[k]:offs[k + 1]].reshape(wl.pairs[k].height, wl.pairs[k].width) for k in order]
        per_np = per.double().cpu().numpy()
        e_or = oracle_spot_check(wl, th_last, xhs, [per_np[k] for k in order], order)
        line["hg_rel_err_oracle"] = {"pairs": order, "errors": e_or,
                                     "ref": "FP64 checker at the GPU's last point, reference solve to 1e-12"}
    if rank == 0 and world == 1 and args.cpu_baseline:
        sec, n, desc = oracle_sample(2, 1, max_seconds=30.0, strategy=args.strategy, workload=args.workload,
                                     variant=args.refresh, method=args.method, rtol=args.rtol)
        k0 = min(range(K), key=lambda k: wl.pairs[k].height * wl.pairs[k].width)
        px0 = wl.pairs[k0].height * wl.pairs[k0].width
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "hypergradients/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc, "pixel_hypergradients_per_s": px0 / sec}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
