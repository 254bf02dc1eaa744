"""Throughput benchmark of the radiation step on GB300.

One bench step = one SSP-RK2 step of the whole hot path (transport in space
and angle, stage update, implicit coupling, n0crit guard; rad_step) plus the
moment contraction (rad_moments) over the 3D turbulent flat-space workload:
128^3 cells x 162 geodesic bins (level 4), periodic, moving gas, seeded
synthetic fields.  The metric is cell-angle updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f64]
                  [--impl ours|reference]

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (the comparison arm; it is a deliberately plain
program).  With N > 1 (torchrun) the domain is N copies of the workload's
periodic 128^3 block laid along x1, one block per GPU: before each RK stage
every rank packs the three cell layers next to its two x1 faces, exchanges
them with its neighbours over NCCL and steps on the received halos (weak
scaling; value is the whole job's cell-angle updates over the slowest
rank's time).  --replicas runs N unconnected copies instead; --decomp-self
runs the one-GPU case through the same pack / exchange / staged path, the
block's x1 faces shared with itself.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "turb3d"
# FP64 arithmetic of one cell-angle update (both RK stages) of the flat PLM
# thermal step, counted from the stage kernel (an FMA as 2, a division as 1),
# per stage: x1 and x2 in the upwind frame, 14 each (three differences, two
# van Leer slopes, the two upwind face states and their weights); x3 from the
# register window, 11 (one new slope, the face pair); the stage combination
# and the sum of the three divergences, 5.5; the coupling sums, 20 (n0bar,
# the weights and the per-bin and warp sums); the implicit update and guard,
# 19; the gas-source terms, 8; ~92 per stage, with the per-cell quartic and
# gas source adding ~1 per update
FLOPS_PER_UPDATE = 184
FP64_PEAK_TFLOPS = 1.25
WORKLOAD_TEXT = ("turb3d: flat-space Cartesian 128^3, geodesic level 4 (162 bins), periodic, moving gas "
                 "|v|<=0.5, log-uniform opacities, PLM, thermal coupling")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--precision", default="f32", choices=["f32", "f64"])
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n", type=int, default=None, help="cells per side (default: the workload's 128)")
    p.add_argument("--workload", default=WORKLOAD, choices=["turb3d", "torus3d", "torus3d_big"],
                   help="the stepped workload: turb3d (the benchmark); the Kerr-Schild ones time and "
                        "profile the curved-space kernels and run only with --no-e2e --no-extras "
                        "--no-cpu-baseline")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP64-path, accuracy and adjoint/forward measurements")
    p.add_argument("--replicas", action="store_true", help="N > 1: unconnected replicas instead of blocks")
    p.add_argument("--decomp-self", action="store_true",
                   help="N = 1: step through the block path, x1 faces shared with the block itself")
    return p.parse_args()


def max_over_ranks(x, device, world):
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds_local, device, world):
    """Whole-job throughput of N replicas: all ranks' units over the slowest
    rank's time."""
    return units_per_rank * max(1, world) / max_over_ranks(seconds_local, device, world)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 100 ms), each stamped with the host clock on
    arrival; summary() keeps those that arrived inside the timed window."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.window = (0.0, float("inf"))

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def ready(self, timeout=10.0):
        """Wait for the first sample: nvidia-smi's start-up must not fall
        inside the timed region."""
        t0 = time.perf_counter()
        while self.proc and not self.rows and time.perf_counter() - t0 < timeout:
            time.sleep(0.05)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        lo, hi = self.window
        rows = [r for (t, r) in self.rows if lo <= t <= hi]
        if not rows:         # window shorter than one sampling period: nearest samples
            rows = [r for (t, r) in sorted(self.rows, key=lambda x: abs(x[0] - 0.5 * (lo + hi)))[:2]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if len(r) > 2)
        mx = max(float(r[2]) for r in rows if len(r) > 2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(rows)}


def setup_gpu(prec, dev, n=None, name=WORKLOAD, block=None):
    """block = (index, count): the block's x1 faces are shared with its
    neighbours along x1 (RAD_BC_HALO) and its x1 coordinates are shifted by
    `index` periods."""
    import torch
    import paper_2302_04283_gb300 as rad
    import workloads as W
    # --n scales the workload's grid: n^3 for the Cartesian box, n x n/2 x n/2
    # (the default aspect) for the Kerr-Schild ones
    shape = None if not n else ((n, n, n) if name == WORKLOAD else (n, n // 2, n // 2))
    w = W.make(name, n=shape, with_intensity=False)
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, w["level"])
    xf, bc = w["xf"], w["bc"]
    if block is not None:
        period = float(xf[0][-1] - xf[0][0])
        xf = [xf[0] + block[0] * period, xf[1], xf[2]]
        bc = (("halo", "halo"), bc[1], bc[2])
    rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], xf, bc)
    dt = rad.rad_cfl_dt(ctx, w["cfl"])
    sh = (w["n"][2], w["n"][1], w["n"][0])
    tdt = torch.float32 if prec == "f32" else torch.float64
    g = torch.Generator(device=dev)
    g.manual_seed(w["seed"])
    T = torch.tensor(w["T"], device=dev)
    B = (T ** 4 / (4 * math.pi))[..., None]
    I = torch.empty(sh + (nap,), dtype=tdt, device=dev)
    I[..., :na] = (B * (1 + 0.1 * (2 * torch.rand(sh + (na,), generator=g, device=dev, dtype=torch.float64) - 1))).to(tdt)
    I[..., na:] = 0
    gas = {k: torch.tensor(np.ascontiguousarray(w[k]), device=dev) for k in ("rho", "u", "alpha_a", "alpha_s")}
    gas["T"] = T
    gas["eta"] = None
    return rad, w, ctx, na, nap, dt, sh, tdt, I, gas


PROFILE = os.path.join(ROOT, "profiles", "k_stage_turb3d_f32.md")


def kernel_fingerprint():
    """Hash of the code lines (comments and blank lines dropped) of the stage
    kernel and its launcher: a profile's counters describe this kernel only
    while the fingerprint it records matches."""
    h = hashlib.sha256()
    for f in ("step_kernel.cuh", "stage_launch.cuh", "step.cu"):
        with open(os.path.join(ROOT, "paper_2302_04283_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//")[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(precision, ncell):
    """DRAM bytes per k_stage launch (average of the two stages) from the
    committed ncu summary, scaled by cells to this grid; None when the
    summary is missing, was taken on another precision, or the kernel has
    changed since."""
    try:
        kv = {}
        with open(PROFILE) as fh:
            for line in fh:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("fingerprint") != kernel_fingerprint() or kv.get("precision") != precision:
            return None
        return float(kv["dram_bytes_per_launch"]) * ncell / float(kv["cells"])
    except Exception:
        return None


def block_step_fn(rad, ctx, I, gas, dt, opts, src, rank, world, nap, tdt, dev, sh):
    """One RK2 step of this rank's block: x1 halos exchanged with the
    neighbouring ranks over torch.distributed (NCCL), or, for one block
    whose faces are shared with itself, copied locally."""
    from paper_2302_04283_gb300 import blocks as B
    nb = {(0, 0): (rank - 1) % world, (0, 1): (rank + 1) % world}
    send, recv = B.halo_buffers(sh, nb, nap, tdt, dev)
    move = None
    if world == 1:
        def move(s_, r_):
            r_[(0, 0)].copy_(s_[(0, 1)])
            r_[(0, 1)].copy_(s_[(0, 0)])

    def step():
        B.step_block(rad, ctx, I, gas, dt, opts, src, nb, send, recv, move)
    return step


def run_ours(args, rank, world):
    import torch
    dev = f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}"
    torch.cuda.set_device(dev)
    blocks = (world > 1 and not args.replicas) or (world == 1 and args.decomp_self)
    rad, w, ctx, na, nap, dt, sh, tdt, I, gas = setup_gpu(args.precision, dev, args.n, name=args.workload,
                                                          block=(rank, world) if blocks else None)
    if blocks and world > 1:
        from paper_2302_04283_gb300 import blocks as B
        dt = B.domain_dt(dt, device=dev)                                        # the domain's bound
    ncell = sh[0] * sh[1] * sh[2]
    esz = 4 if args.precision == "f32" else 8
    prec = rad.RAD_F32 if args.precision == "f32" else rad.RAD_F64
    mom = rad.RAD_MOM_BF16X3 if args.precision == "f32" else rad.RAD_MOM_SIMT
    opts = rad.rad_opts_default(precision=prec)
    src = torch.zeros(sh + (4,), dtype=torch.float64, device=dev)
    R = torch.zeros(sh + (10,), dtype=tdt, device=dev)
    I0 = I.clone()
    T0 = gas["T"].clone()
    st = torch.cuda.current_stream()

    advance = (block_step_fn(rad, ctx, I, gas, dt, opts, src, rank, world, nap, tdt, dev, sh) if blocks
               else (lambda: rad.rad_step(ctx, I, gas, dt, opts, src)))

    def step(ev=None):
        if ev:
            ev[0].record(st)
        advance()
        if ev:
            ev[1].record(st)
        rad.rad_moments(ctx, I, prec, rad.RAD_FRAME_TETRAD, mom, gas, R)
        if ev:
            ev[2].record(st)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        clk.ready()
        for _ in range(args.warmup):
            step()
        rad.rad_check(ctx)
        # reset the state so every run times the same steps of the same workload
        I.copy_(I0)
        gas["T"].copy_(T0)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        start.record(st)
        for s in range(args.steps):
            step(evs[s])
        stop.record(st)
        torch.cuda.synchronize()
        clk.window = (t0, time.perf_counter())
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(stop)
    stage_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
    mom_ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    rad.rad_check(ctx)
    value = job_rate(ncell * na * args.steps, total_ms * 1e-3, dev, world)
    total_ms = max_over_ranks(total_ms, dev, world)
    # algorithmic bytes of the two stage launches of one step (per cell-angle:
    # stage 1 reads I^0, writes I^1; stage 2 reads I^1 and I^0, writes I^2;
    # per cell: gas fields rho, u(3), alpha_a, alpha_s and T in/out, the
    # stage temperature, and the 4-vector source)
    bytes_step = ncell * na * 5 * esz + ncell * 8 * (6 + 2 + 2 + 1 + 4 + 4)
    achieved = bytes_step * args.steps / (stage_ms * 1e-3) / 1e9
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    traffic = profiled_traffic(args.precision, ncell) if args.workload == WORKLOAD else None
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm or 6800.0,
            "unit": "GB/s", "frac": round(achieved / (hbm or 6800.0), 4),
            "traffic": None if traffic is None else round(traffic),
            "kernel": "k_stage (per launch: mean of the stage-1 and stage-2 launches)",
            "algorithmic_bytes_per_launch": bytes_step // 2,
            "peak_source": "measured" if hbm else "fallback"}
    if args.precision == "f64":
        # the FP64 path is bound by the FP64 pipe: rate against GB300's nominal
        # 1.25 TFLOP/s FP64 (FMA = 2 flops, a division counted as 1)
        tflops = FLOPS_PER_UPDATE * ncell * na * args.steps / (stage_ms * 1e-3) / 1e12
        meas = rad.rad_fp64_fma_rate(3.0)
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(tflops / FP64_PEAK_TFLOPS, 4), "traffic": None,
                "kernel": "k_stage (both stages)", "flops_per_update": FLOPS_PER_UPDATE,
                "peak_source": "nominal FP64 rate", "hbm_achieved_gbs": round(achieved, 1),
                "peak_measured": round(meas, 4), "frac_of_measured": round(tflops / meas, 4),
                "peak_measured_source": "rad_fp64_fma_rate: DFMA chains on every SM, CUDA events"}
    res = {
        "metric": "cell-angle updates/sec", "value": value, "unit": "cell-angle updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "f32" else "f64",
        "data": ("synthetic (seeded turbulent-gas workload; no dataset in the paper)" if args.workload == WORKLOAD
                 else "synthetic (seeded torus-gas workload; no dataset in the paper)"),
        "config": {"workload": WORKLOAD_TEXT if args.workload == WORKLOAD else
                   f"{args.workload}: Kerr-Schild a={w['spin']}, {w['n'][0]}x{w['n'][1]}x{w['n'][2]} cells, "
                   f"geodesic level {w['level']} ({na} bins)",
                   "cells": ncell, "bins": na, "precision": args.precision,
                   "moments": "split-bf16 tensor cores" if mom == rad.RAD_MOM_BF16X3 else "CUDA cores",
                   "l2": "inputs larger than L2 (I is %.2f GB), no flush" % (ncell * nap * esz / 1e9),
                   "parallelism": (f"x1 blocks x{world}, 128^3 cells per GPU, ghost exchange before each stage "
                                   f"({'NCCL' if world > 1 else 'the block with itself'})") if blocks
                                  else f"replicas x{world}"},
        "roofline": roof,
        "gpu_launches": (7 if blocks else 3) * args.steps,
        "clocks": clk.summary(),
        "breakdown_ms_per_step": {"rad_step": stage_ms / args.steps, "rad_moments": mom_ms / args.steps,
                                  "step_min": min(step_ms), "step_median": sorted(step_ms)[len(step_ms) // 2],
                                  "step_max": max(step_ms)},
    }
    if not args.no_e2e:
        if blocks:
            res["e2e"] = run_e2e_blocks(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world, rank)
        else:
            res["e2e"] = run_e2e(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world)
    rad.rad_destroy(ctx)
    if not args.no_extras and world == 1 and args.precision == "f32":
        res["extras"] = run_extras(args, dev)
    return res


def _time_steps(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


GOLDEN = os.path.join(ROOT, "tests", "golden")


def config_errors(dev):
    """Error of each precision against the FP64 oracle's stored values
    (tests/golden, written by oracle-only scripts) for the 3D workloads at
    their full sizes and stated step counts: normwise (max |d| / max |ref|)
    and per element (max |d| / |ref|) for sampled intensities and T, and
    max |d| / R^00 for the moments."""
    import torch
    import paper_2302_04283_gb300 as rad
    import workloads as W
    out = {}
    for name, fname in (("turb3d", "turb3d_samples.npz"), ("torus3d", "torus3d_samples.npz"),
                        ("torus3d_big", "torus3d_big_subvolume.npz")):
        path = os.path.join(GOLDEN, fname)
        if not os.path.exists(path):
            out[name] = "no stored oracle values"
            continue
        g = np.load(path)
        w = W.make(name, with_intensity=False)
        ctx = rad.rad_create(torch.cuda.current_stream())
        na, nap = rad.rad_init_angles(ctx, w["level"])
        gdir, _, _ = rad.rad_get_angles(ctx, na)
        rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], w["xf"], w["bc"])
        # the stored values' bin order -> this library's bins (same directions)
        odir = g["dirs"]
        gmap = ((odir[:, None, :] - gdir[None, :, :]) ** 2).sum(-1).argmin(1)
        if sorted(gmap.tolist()) != list(range(na)):
            raise RuntimeError("stored bin directions do not match this grid")
        n1, n2, n3 = w["n"]
        dt = float(g["dt"])
        res = {"steps": int(g["steps"]), "cells": n1 * n2 * n3, "bins": na}
        for prec, method in (("f64", rad.RAD_MOM_SIMT), ("f32+bf16", rad.RAD_MOM_BF16X3)):
            f32 = prec != "f64"
            tdt = torch.float32 if f32 else torch.float64
            I = torch.zeros((n3, n2, n1, nap), dtype=tdt, device=dev)
            for k in range(n3):
                row = np.zeros((n2, n1, nap))
                row[..., gmap] = W.intensity_rows(w, k)
                I[k] = torch.tensor(row, device=dev).to(tdt)
            t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
            gas = {k: t(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s", "T")}
            gas["eta"] = None
            o = rad.rad_opts_default(precision=rad.RAD_F32 if f32 else rad.RAD_F64)
            for _ in range(int(g["steps"])):
                rad.rad_step(ctx, I, gas, dt, o)
            R = torch.zeros((n3, n2, n1, 10), dtype=tdt, device=dev)
            rad.rad_moments(ctx, I, o.precision, rad.RAD_FRAME_TETRAD, method, gas, R)
            torch.cuda.synchronize()
            rad.rad_check(ctx)
            if name == "torus3d_big":
                i0, j0, k0 = (int(x) for x in g["origin"])
                S = int(g["sub"])
                kk = torch.tensor(np.arange(k0, k0 + S) % n3, device=dev)
                sub = lambda X: X[kk][:, j0:j0 + S, i0:i0 + S]
                Tg, Rg = sub(gas["T"]).cpu().numpy(), sub(R).double().cpu().numpy()
                c = g["sample_cells"]
                Ig = sub(I).double().cpu().numpy()[c[:, 0], c[:, 1], c[:, 2]][np.arange(len(c)), gmap[g["sample_bins"]]]
                To, Ro, Io = g["T"], g["R"], g["sample_I"]
            else:
                c, bc = g["cells"], g["bin_cells"]
                Tg = gas["T"].cpu().numpy()[c[:, 0], c[:, 1], c[:, 2]]
                Rg = R.double().cpu().numpy()[c[:, 0], c[:, 1], c[:, 2]]
                Ig = I[torch.tensor(bc[:, 0]), torch.tensor(bc[:, 1]), torch.tensor(bc[:, 2]),
                       torch.tensor(gmap[g["bins"]])].double().cpu().numpy()
                To, Ro, Io = g["T"], g["R"], g["I"]

            def errs(a_, b_):
                d = np.abs(a_ - b_)
                return {"normwise": float(d.max() / np.abs(b_).max()),
                        "per_element": float((d / np.maximum(np.abs(b_), 1e-300)).max())}
            res[prec] = {"I": errs(Ig, Io), "T": errs(Tg, To),
                         "R_over_R00": float((np.abs(Rg - Ro) / np.abs(Ro[..., :1])).max())}
            del I, R
        res["stated_tolerance"] = {"f64": 1e-12, "f32 (I, T)": 2e-5, "bf16 moments (of R^00)": 1.5e-4}
        rad.rad_destroy(ctx)
        out[name] = res
    return out


def run_extras(args, dev):
    """Measurements that complete the metric: the plain FP64 path on the same
    workload, the FP32 / split-BF16 error against the FP64 path after one step
    (the FP64 path matches the FP64 oracle to 1e-12, a parity test), and the
    adjoint/forward time ratio on the 2D Kerr-Schild adjoint workload."""
    import torch
    out = {}
    out["vs_oracle_at_stated_steps"] = config_errors(dev)
    rad, w, ctx, na, nap, dt, sh, _, I32, gas = setup_gpu("f32", dev, args.n)
    I64 = torch.zeros(sh + (nap,), dtype=torch.float64, device=dev)
    I64[..., :na] = I32[..., :na].double()
    T0 = gas["T"].clone()
    ncell = sh[0] * sh[1] * sh[2]
    o64 = rad.rad_opts_default(precision=rad.RAD_F64)
    o32 = rad.rad_opts_default(precision=rad.RAD_F32)
    # plain FP64 path, same workload
    Rb = torch.zeros(sh + (10,), dtype=torch.float64, device=dev)

    def s64():
        rad.rad_step(ctx, I64, gas, dt, o64)
        rad.rad_moments(ctx, I64, rad.RAD_F64, rad.RAD_FRAME_TETRAD, rad.RAD_MOM_SIMT, gas, Rb)

    gas["T"].copy_(T0)
    ms64 = _time_steps(s64, 3, 1)
    rad.rad_check(ctx)
    fp64_tf = FLOPS_PER_UPDATE * ncell * na / (ms64 * 1e-3) / 1e12
    fp64_meas = rad.rad_fp64_fma_rate(3.0)
    out["f64_plain"] = {"value": ncell * na / (ms64 * 1e-3), "unit": "cell-angle updates/s", "ms_per_step": ms64,
                        "fp64_tflops": fp64_tf,
                        "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                        "fp64_peak_tflops_measured": round(fp64_meas, 4),
                        "frac_of_measured_fp64": round(fp64_tf / fp64_meas, 4),
                        "what": "rad_step FP64 + rad_moments FP64 on CUDA cores, same workload, 3 steps; "
                                "peak measured live by rad_fp64_fma_rate (DFMA chains on every SM)"}
    rad.rad_destroy(ctx)
    del I64, I32, Rb
    # the Kerr-Schild workloads (angular fluxes, polar and outflow boundaries)
    for name in ("torus3d", "torus3d_big"):
        rad, w, ctx, na, nap, dt, sh, _, Ik, gk = setup_gpu("f32", dev, None, name)
        Rk = torch.zeros(sh + (10,), dtype=torch.float32, device=dev)

        def sk():
            rad.rad_step(ctx, Ik, gk, dt, o32)
            rad.rad_moments(ctx, Ik, rad.RAD_F32, rad.RAD_FRAME_TETRAD, rad.RAD_MOM_BF16X3, gk, Rk)

        msk = _time_steps(sk, 3, 1)
        rad.rad_check(ctx)
        ncell_k = sh[0] * sh[1] * sh[2]
        out[name + "_f32"] = {"value": ncell_k * na / (msk * 1e-3), "unit": "cell-angle updates/s",
                              "ms_per_step": msk, "cells": ncell_k, "bins": na,
                              "what": "rad_step FP32 + split-BF16 moments, 3 steps, Kerr-Schild a=0.9"}
        rad.rad_destroy(ctx)
        del Ik, Rk, gk
    # adjoint / forward on the adjoint workload (FP64, fixed emissivity)
    import workloads as W
    wa = W.make("adjoint2d", with_intensity=False)
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, wa["level"])
    rad.rad_set_metric(ctx, wa["kind"], wa["spin"], wa["ndim"], wa["xf"], wa["bc"])
    dta = rad.rad_cfl_dt(ctx, wa["cfl"])
    sha = (wa["n"][2], wa["n"][1], wa["n"][0])
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    gA = {k: t(wa[k]) for k in ("rho", "u", "alpha_a", "alpha_s", "eta", "T")}
    oa = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
    Ia = torch.full(sha + (nap,), 1.0 / (4 * math.pi), dtype=torch.float64, device=dev)
    Ia[..., na:] = 0
    lam = torch.ones_like(Ia)
    lam_n = torch.empty_like(Ia)
    ga, gs, ge = (torch.zeros(sha, dtype=torch.float64, device=dev) for _ in range(3))
    Iw = Ia.clone()
    fwd = _time_steps(lambda: rad.rad_step(ctx, Iw, gA, dta, oa), 8, 2)
    adj = _time_steps(lambda: rad.rad_step_adjoint(ctx, Ia, gA, dta, oa, lam, lam_n, None, None, ga, gs, ge), 8, 2)
    # the same in FP32
    o32 = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_EMISSIVITY)
    Ia32, lam32 = Ia.float(), lam.float()
    lam_n32, Iw32 = torch.empty_like(Ia32), Ia32.clone()
    fwd32 = _time_steps(lambda: rad.rad_step(ctx, Iw32, gA, dta, o32), 8, 2)
    adj32 = _time_steps(lambda: rad.rad_step_adjoint(ctx, Ia32, gA, dta, o32, lam32, lam_n32, None, None, ga, gs, ge), 8, 2)
    # thermal coupling (gradient through the quartic and the temperature), FP64
    oth = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_THERMAL)
    gT = dict(gA, eta=None)
    Tw = gT["T"].clone()
    gTw = dict(gT, T=Tw)
    lamT, lamT_n = torch.ones_like(Tw), torch.empty_like(Tw)
    fwdT = _time_steps(lambda: rad.rad_step(ctx, Iw, gTw, dta, oth), 8, 2)
    adjT = _time_steps(lambda: rad.rad_step_adjoint(ctx, Ia, gT, dta, oth, lam, lam_n, lamT, lamT_n, ga, gs, None),
                       8, 2)
    rad.rad_check(ctx)
    rad.rad_destroy(ctx)
    out["adjoint_over_forward"] = {"ratio": adj / fwd, "fwd_ms_per_step": fwd, "adj_ms_per_step": adj,
                                   "ratio_f32": adj32 / fwd32, "fwd_ms_per_step_f32": fwd32,
                                   "adj_ms_per_step_f32": adj32,
                                   "ratio_thermal": adjT / fwdT, "fwd_ms_per_step_thermal": fwdT,
                                   "adj_ms_per_step_thermal": adjT,
                                   "workload": "adjoint2d: Kerr-Schild a=0.5, 256x128, level 4 (162 bins), "
                                               "fixed-emissivity coupling (ratio, ratio_f32) and thermal coupling "
                                               "(ratio_thermal, FP64); adjoint includes the recomputation"}
    return out


def run_e2e(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world):
    """Same metric through the public host-buffer API (rad_step_host): every
    step copies its inputs (I and the gas state) from pinned host memory,
    steps, contracts and reads the moments and temperature back; the library
    overlaps one step's copies with the neighbouring step's kernels."""
    import torch
    import workloads as W
    w = W.make(WORKLOAD, n=(sh[2], sh[1], sh[0]), with_intensity=False)
    hI = torch.empty(sh + (nap,), dtype=tdt, pin_memory=True)
    g = torch.Generator()
    g.manual_seed(w["seed"])
    T = torch.tensor(w["T"])
    hI[..., :na] = ((T ** 4 / (4 * math.pi))[..., None] *
                    (1 + 0.1 * (2 * torch.rand(sh + (na,), generator=g, dtype=torch.float64) - 1))).to(tdt)
    hI[..., na:] = 0
    hgas = {k: torch.tensor(np.ascontiguousarray(w[k])).pin_memory() for k in ("rho", "u", "alpha_a", "alpha_s")}
    # one item per step; the temperature is copied in and out on every step.
    # Items in flight together must not share output buffers, so three
    # (temperature, moments) pairs rotate; the read-only inputs are shared.
    items = []
    for _ in range(3):
        hT = torch.tensor(np.ascontiguousarray(w["T"])).pin_memory()
        hR = torch.empty(sh + (10,), dtype=tdt, pin_memory=True)
        items.append(dict(hgas, I=hI, eta=None, T=hT, R=hR))
    seq = lambda n: [items[q % len(items)] for q in range(n)]
    # this machine's sustained pinned host-to-device rate (four back-to-back
    # copies of the intensity array, just before and just after the timed
    # region): the step rate the uploads alone allow.  The sustained rate of
    # the host link varies over time on a shared machine (a single copy does
    # not show it), so both ends are reported.
    dI = torch.empty_like(hI, device=dev)
    s = torch.cuda.current_stream()

    def link_gbs(n=4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dI.copy_(hI, non_blocking=True)
        e0.record(s)
        for _ in range(n):
            dI.copy_(hI, non_blocking=True)
        e1.record(s)
        torch.cuda.synchronize()
        return n * hI.numel() * hI.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9

    rad.rad_step_host(ctx, seq(max(1, args.warmup)), dt, opts, 1, rad.RAD_FRAME_TETRAD, mom)
    gbs_before = link_gbs()
    t0 = time.perf_counter()
    rad.rad_step_host(ctx, seq(args.steps), dt, opts, 1, rad.RAD_FRAME_TETRAD, mom)
    el = time.perf_counter() - t0
    h2d_gbs = link_gbs()
    del dI
    rate = job_rate(sh[0] * sh[1] * sh[2] * na * args.steps, el, dev, world)
    h2d = hI.numel() * hI.element_size() + sum(v.numel() * v.element_size() for v in hgas.values()) + \
        hT.numel() * hT.element_size()
    d2h = hR.numel() * hR.element_size() + hT.numel() * hT.element_size()
    return {"value": rate, "unit": "cell-angle updates/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "h2d_gbs_measured": round(h2d_gbs, 1), "h2d_gbs_before": round(gbs_before, 1),
            # the rate the uploads alone allow at the better of the two link
            # measurements (what the link showed it can sustain)
            "upload_bound_value": sh[0] * sh[1] * sh[2] * na / (h2d / (max(h2d_gbs, gbs_before) * 1e9)),
            "api": "rad_step_host (host buffers; uploads, read-backs and moments on their own streams, overlapping the steps)",
            "reads_back": "the step's results: moments R^{AB} [cell][10] and gas temperature T [cell]; the evolved "
                          "intensity stays on the device (rad_host_item.I_out is null)"}


def run_e2e_blocks(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world, rank):
    """End to end for the block path: every step copies this rank's block
    (I and the gas state) from pinned host memory, steps it with the ghost
    exchange, contracts the moments and reads the moments and temperature
    back (one stream, no overlap)."""
    import torch
    import workloads as W
    w = W.make(WORKLOAD, n=(sh[2], sh[1], sh[0]), with_intensity=False)
    hI = torch.empty(sh + (nap,), dtype=tdt, pin_memory=True)
    g = torch.Generator()
    g.manual_seed(w["seed"])
    T = torch.tensor(w["T"])
    hI[..., :na] = ((T ** 4 / (4 * math.pi))[..., None] *
                    (1 + 0.1 * (2 * torch.rand(sh + (na,), generator=g, dtype=torch.float64) - 1))).to(tdt)
    hI[..., na:] = 0
    hgas = {k: torch.tensor(np.ascontiguousarray(w[k])).pin_memory() for k in ("rho", "u", "alpha_a", "alpha_s", "T")}
    hR = torch.empty(sh + (10,), dtype=tdt, pin_memory=True)
    hT = torch.empty(sh, dtype=torch.float64, pin_memory=True)
    dI = torch.empty(sh + (nap,), dtype=tdt, device=dev)
    dgas = {k: torch.empty_like(v, device=dev) for k, v in hgas.items()}
    dgas["eta"] = None
    dR = torch.empty(sh + (10,), dtype=tdt, device=dev)
    src = torch.zeros(sh + (4,), dtype=torch.float64, device=dev)
    step = block_step_fn(rad, ctx, dI, dgas, dt, opts, src, rank, world, nap, tdt, dev, sh)

    def one():
        dI.copy_(hI, non_blocking=True)
        for k, v in hgas.items():
            dgas[k].copy_(v, non_blocking=True)
        step()
        rad.rad_moments(ctx, dI, prec, rad.RAD_FRAME_TETRAD, mom, dgas, dR)
        hR.copy_(dR, non_blocking=True)
        hT.copy_(dgas["T"], non_blocking=True)

    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    rate = job_rate(sh[0] * sh[1] * sh[2] * na * args.steps, el, dev, world)
    h2d = hI.numel() * hI.element_size() + sum(v.numel() * v.element_size() for v in hgas.values())
    d2h = hR.numel() * hR.element_size() + hT.numel() * hT.element_size()
    return {"value": rate, "unit": "cell-angle updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "blocks.step_block (rad_halo_pack, exchange, rad_step_stage) + rad_moments, host buffers "
                   "copied in and out every step on one stream",
            "reads_back": "moments R^{AB} [cell][10] and gas temperature T [cell] of this rank's block"}


# ------------------------------------------------------- oracle on CPU
class OracleSample:
    """The FP64 oracle on a bounded sample of the workload: the same recipe on
    an n-cell periodic block (setup excluded from timing)."""

    def __init__(self, n=(24, 24, 24)):
        import torch
        import workloads as W
        from oracle import cfl as OCFL
        from oracle.angles import GeodesicGrid
        from oracle.transport import Grid, Setup
        from oracle import step as OS
        self.n = n
        w = W.make(WORKLOAD, n=n)
        self.ang = GeodesicGrid(w["level"])
        self.st = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), self.ang)
        self.dt = OCFL.cfl_dt(self.st, w["cfl"])
        self.gas = {k: torch.tensor(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s")}
        self.gas["eta"] = None
        self.I, self.T = torch.tensor(w["I0"]), torch.tensor(w["T"])
        self.opts = OS.Opts()
        self.cells = n[0] * n[1] * n[2]

    def step(self):
        from oracle import moments as OM
        from oracle import step as OS
        self.I, self.T, _, _ = OS.rk2_step(self.I, self.T, self.gas, self.dt, self.st, self.opts)
        OM.moments(self.I, self.ang)

    def describe(self, steps, el):
        import torch
        return {"value": self.cells * self.ang.n_ang * steps / el, "unit": "cell-angle updates/s",
                "cores": torch.get_num_threads(), "threads": torch.get_num_threads(),
                "host_cpus": os.cpu_count(), "kind": "oracle",
                "sample": f"{self.n[0]}x{self.n[1]}x{self.n[2]} cells x {self.ang.n_ang} bins of the turb3d "
                          f"recipe, {steps} RK2 steps + moments, FP64 ({el:.1f} s timed)"}


def oracle_sample(steps=40):
    """The oracle's rate in a fresh process (the same code path as the
    reference arm, so the two numbers differ only by their samples' noise)."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", str(steps),
           "--warmup", "3"]
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    return json.loads(line)["cpu_baseline"]


def run_reference(args):
    import torch
    torch.set_num_threads(os.cpu_count() or 1)
    o = OracleSample()
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    el = time.perf_counter() - t0
    info = o.describe(args.steps, el)
    v = info["value"]
    return {"impl": "reference", "metric": "cell-angle updates/sec", "value": v, "unit": "cell-angle updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded turbulent-gas workload; no dataset in the paper)",
            "config": {"workload": WORKLOAD_TEXT if args.workload == WORKLOAD else
                   f"{args.workload}: Kerr-Schild a={w['spin']}, {w['n'][0]}x{w['n'][1]}x{w['n'][2]} cells, "
                   f"geodesic level {w['level']} ({na} bins)", "cells": 128 ** 3, "bins": 162,
                       "sample": f"each step advances a {o.n[0]}^3-cell block of the same recipe (bounded CPU "
                                 "work); the rate is per cell-angle update, comparable with the GPU arm"},
            "cpu_baseline": info, "e2e": {"value": v, "unit": "cell-angle updates/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.workload != WORKLOAD and not (args.no_e2e and args.no_extras and args.no_cpu_baseline):
        raise SystemExit("--workload other than turb3d runs only with --no-e2e --no-extras --no-cpu-baseline")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import datetime
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        # a bounded timeout: a rank that stops answering ends the job with an
        # error instead of holding every GPU
        torch.distributed.init_process_group("nccl", timeout=datetime.timedelta(seconds=300))
    res = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = oracle_sample()
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
