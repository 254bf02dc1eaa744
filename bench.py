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
program).  With N > 1 (torchrun) every rank runs an independent replica of
the workload on its own GPU (no halo exchange is built), and value is the
sum over ranks.
"""
import argparse
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--precision", default="f32", choices=["f32", "f64"])
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n", type=int, default=None, help="cells per side (default: the workload's 128)")
    return p.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- our arm
def setup_gpu(prec, dev, n=None):
    import torch
    import paper_2302_04283_gb300 as rad
    import workloads as W
    w = W.make(WORKLOAD, n=(n, n, n) if n else None, with_intensity=False)
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, w["level"])
    rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], w["xf"], w["bc"])
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


def run_ours(args, rank, world):
    import torch
    dev = f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}"
    torch.cuda.set_device(dev)
    rad, w, ctx, na, nap, dt, sh, tdt, I, gas = setup_gpu(args.precision, dev, args.n)
    ncell = sh[0] * sh[1] * sh[2]
    esz = 4 if args.precision == "f32" else 8
    prec = rad.RAD_F32 if args.precision == "f32" else rad.RAD_F64
    mom = rad.RAD_MOM_BF16X3 if args.precision == "f32" else rad.RAD_MOM_SIMT
    opts = rad.rad_opts_default(precision=prec)
    src = torch.zeros(sh + (4,), dtype=torch.float64, device=dev)
    R = torch.zeros(sh + (10,), dtype=tdt, device=dev)
    I0 = I.clone()
    T0 = gas["T"].clone()
    try:
        rad.rad_moments(ctx, I, prec, rad.RAD_FRAME_TETRAD, mom, gas, R)
    except rad.RadError:
        mom = rad.RAD_MOM_SIMT
    st = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(st)
        rad.rad_step(ctx, I, gas, dt, opts, src)
        if ev:
            ev[1].record(st)
        rad.rad_moments(ctx, I, prec, rad.RAD_FRAME_TETRAD, mom, gas, R)
        if ev:
            ev[2].record(st)

    for _ in range(args.warmup):
        step()
    rad.rad_check(ctx)
    # reset the state so every run times the same steps of the same workload
    I.copy_(I0)
    gas["T"].copy_(T0)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        start.record(st)
        for s in range(args.steps):
            step(evs[s])
        stop.record(st)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(stop)
    stage_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
    mom_ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    rad.rad_check(ctx)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    updates = ncell * na * args.steps * world
    value = updates / (total_ms * 1e-3)
    # algorithmic bytes of the two stage launches of one step (per cell-angle:
    # stage 1 reads I^0, writes I^1; stage 2 reads I^1 and I^0, writes I^2;
    # per cell: gas fields rho, u(3), alpha_a, alpha_s and T in/out, the
    # stage temperature, and the 4-vector source)
    bytes_stage = ncell * na * 5 * esz + ncell * 8 * (6 + 2 + 2 + 1 + 4 + 4)
    achieved = bytes_stage * args.steps / (stage_ms * 1e-3) / 1e9
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm or 6800.0,
            "unit": "GB/s", "frac": round(achieved / (hbm or 6800.0), 4),
            "traffic": None, "kernel": "k_stage (both RK2 stages)",
            "peak_source": "measured" if hbm else "fallback"}
    if args.precision == "f64":
        roof["note"] = "FP64 path: bound by the FP64 pipe (see DESIGN.md), HBM fraction shown for reference"
    res = {
        "metric": "cell-angle updates/sec", "value": value, "unit": "cell-angle updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "f32" else "f64",
        "data": "synthetic (seeded turbulent-gas workload; no dataset in the paper)",
        "config": {"workload": "turb3d: flat-space Cartesian 128^3, geodesic level 4 (162 bins), periodic, "
                               "moving gas |v|<=0.5, log-uniform opacities, PLM, thermal coupling",
                   "cells": ncell, "bins": na, "precision": args.precision,
                   "moments": "split-bf16 tensor cores" if mom == rad.RAD_MOM_BF16X3 else "CUDA cores",
                   "l2": "inputs larger than L2 (I is %.2f GB)" % (ncell * nap * esz / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "breakdown_ms_per_step": {"rad_step": stage_ms / args.steps, "rad_moments": mom_ms / args.steps},
    }
    if not args.no_e2e:
        res["e2e"] = run_e2e(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world)
    rad.rad_destroy(ctx)
    return res


def run_e2e(args, rad, ctx, dt, opts, prec, mom, sh, na, nap, tdt, dev, world):
    """Same metric through the public API with host buffers: every step copies
    its inputs (I and the gas state) from pinned host memory and reads the
    moments back."""
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
    dI = torch.empty_like(hI, device=dev)
    dgas = {k: torch.empty_like(v, device=dev) for k, v in hgas.items()}
    dgas["eta"] = None
    R = torch.empty(sh + (10,), dtype=tdt, device=dev)
    hR = torch.empty(sh + (10,), dtype=tdt, pin_memory=True)
    src = torch.zeros(sh + (4,), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()

    def step():
        dI.copy_(hI, non_blocking=True)
        for k, v in hgas.items():
            dgas[k].copy_(v, non_blocking=True)
        rad.rad_step(ctx, dI, dgas, dt, opts, src)
        rad.rad_moments(ctx, dI, prec, rad.RAD_FRAME_TETRAD, mom, dgas, R)
        hR.copy_(R, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = hI.numel() * hI.element_size() + sum(v.numel() * v.element_size() for v in hgas.values())
    d2h = hR.numel() * hR.element_size()
    ncell = sh[0] * sh[1] * sh[2]
    return {"value": ncell * na * args.steps * world / (ms * 1e-3), "unit": "cell-angle updates/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


# ------------------------------------------------------- oracle on CPU
class OracleSample:
    """The FP64 oracle on a bounded sample of the workload: the same recipe on
    an n-cell periodic block (setup excluded from timing)."""

    def __init__(self, n=(16, 16, 16)):
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
                "cores": torch.get_num_threads(), "kind": "oracle",
                "sample": f"{self.n[0]}x{self.n[1]}x{self.n[2]} cells x {self.ang.n_ang} bins of the turb3d "
                          f"recipe, {steps} RK2 steps + moments, FP64 ({el:.1f} s timed)"}


def oracle_sample(steps=30):
    o = OracleSample()
    o.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    return o.describe(steps, time.perf_counter() - t0)


def run_reference(args):
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
            "data": "synthetic (seeded turbulent-gas workload)",
            "config": {"workload": "turb3d recipe, 16^3-cell sample x 162 bins per step (FP64 CPU oracle)"},
            "cpu_baseline": info, "e2e": {"value": v, "unit": "cell-angle updates/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = oracle_sample()
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
