"""Expected values of the large Kerr-Schild workload after its 20 RK2 steps,
on the 24^3 subvolume centred at r ~ 10, theta = pi/2, phi = 0, written by
the FP64 oracle alone (test infrastructure; nothing here comes from the CUDA
path).

Workload: torus3d_big, Kerr-Schild a = 0.9, 192 x 96 x 96 cells (r log on
[1.5, 50], full theta and phi), geodesic level 8 (642 bins), torus gas with
random velocities <= 0.3c, alpha_s = alpha_a / 2, thermal coupling, PLM,
the n0crit guard, dt = 0.3 x the oracle's time-step bound.

The oracle advances the window of the subvolume plus `margin` cells on every
side (cut with outflow boundaries: wrong values at the cut travel inward
within the numerical domain of dependence, two cells per RK stage with
weights that fall with the Courant number); it does so for two margins and
records their largest difference over the subvolume, which bounds the
truncation error (margins of 8 and 12 cells still differed by 4e-11
relative; 12 and 16 are used).
The time step is the oracle's bound over every (r, theta) column (the
metric does not depend on phi, so one phi slab gives the full grid's bound).

    python tests/golden/make_torus3d_big_subvolume.py [--margins 12 16]

writes tests/golden/torus3d_big_subvolume.npz: R (tetrad-frame moments
[24, 24, 24, 10]), T [24, 24, 24], src (gas source of the last step
[24, 24, 24, 4]), I at 8192 seeded (cell, bin) samples (oracle bin order),
the window, dt, steps, the margin difference and the oracle grid's bin
directions.
"""
import argparse
import math
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import cfl as OCFL  # noqa: E402
from oracle import moments as OM  # noqa: E402
from oracle import step as OS  # noqa: E402
from oracle.angles import GeodesicGrid  # noqa: E402
from oracle.transport import Grid, Setup  # noqa: E402

SUB = 24
STEPS = 20
NSAMPLE = 8192


def subvolume(w):
    """Index ranges (i0, j0, k0) of the 24^3 subvolume: r nearest 10, theta
    around pi/2, phi around 0 (k0 negative: wraps)."""
    rc = 0.5 * (w["xf"][0][1:] + w["xf"][0][:-1])
    ic = int(np.argmin(np.abs(rc - 10.0)))
    n2 = w["n"][1]
    return ic - SUB // 2, n2 // 2 - SUB // 2, -SUB // 2


def window(w, origin, margin):
    """Cell index lists and face coordinates of subvolume + margin."""
    n1, n2, n3 = w["n"]
    i0, j0, k0 = origin
    ii = np.arange(i0 - margin, i0 + SUB + margin)
    jj = np.arange(j0 - margin, j0 + SUB + margin)
    kk = np.arange(k0 - margin, k0 + SUB + margin)
    assert ii.min() >= 0 and ii.max() < n1 and jj.min() >= 0 and jj.max() < n2
    dphi = float(w["xf"][2][1] - w["xf"][2][0])
    xf = [w["xf"][0][ii.min():ii.max() + 2], w["xf"][1][jj.min():jj.max() + 2],
          dphi * np.arange(kk.min(), kk.max() + 2)]
    return ii, jj, kk % n3, xf


def run(w, ang, origin, margin, dt):
    ii, jj, kk, xf = window(w, origin, margin)
    st = Setup(Grid(w["kind"], w["spin"], xf, (("outflow", "outflow"),) * 3, 3), ang)
    cut = lambda a: torch.tensor(np.ascontiguousarray(a[np.ix_(kk, jj, ii)]))
    gas = {key: cut(w[key]) for key in ("rho", "u", "alpha_a", "alpha_s")}
    gas["eta"] = None
    I = torch.tensor(np.stack([np.stack([W.intensity_rows(w, int(k), int(j))[ii] for j in jj]) for k in kk]))
    T = cut(w["T"])
    src = None
    for s in range(STEPS):
        t0 = time.time()
        I, T, src, ok = OS.rk2_step(I, T, gas, dt, st, OS.Opts())
        assert bool(ok.all())
        print(f"  margin {margin}: step {s + 1}/{STEPS} {time.time() - t0:.1f} s", flush=True)
    c = slice(margin, margin + SUB)
    return I[c, c, c], T[c, c, c], src[c, c, c]


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--margins", type=int, nargs=2, default=[12, 16])
    p.add_argument("--out", default=os.path.join(HERE, "torus3d_big_subvolume.npz"))
    a = p.parse_args()
    w = W.make("torus3d_big", with_intensity=False)
    ang = GeodesicGrid(w["level"])
    # the time-step bound over every (r, theta) column: one phi slab
    xf1 = [w["xf"][0], w["xf"][1], w["xf"][2][:2]]
    bc1 = (w["bc"][0], w["bc"][1], ("periodic", "periodic"))
    dt = OCFL.cfl_dt(Setup(Grid(w["kind"], w["spin"], xf1, bc1, 3), ang), w["cfl"])
    print("dt", dt, flush=True)
    origin = subvolume(w)
    res = [run(w, ang, origin, m, dt) for m in a.margins]
    (I, T, src), (I2, T2, src2) = res
    diff = max(float((I - I2).abs().max() / I2.abs().max()), float((T - T2).abs().max() / T2.abs().max()))
    print("margin difference (relative)", diff, flush=True)
    assert diff < 1e-13, diff
    R = OM.moments(I2, ang)
    rng = np.random.default_rng(20)
    cells = rng.integers(0, SUB, (NSAMPLE, 3))
    bins = rng.integers(0, ang.n_ang, NSAMPLE)
    vals = I2.numpy()[cells[:, 0], cells[:, 1], cells[:, 2], bins]
    np.savez_compressed(a.out, R=R.numpy(), T=T2.numpy(), src=src2.numpy(), sample_cells=cells,
                        sample_bins=bins, sample_I=vals, origin=np.array(origin), sub=SUB, steps=STEPS,
                        dt=dt, margins=np.array(a.margins), margin_diff=diff, dirs=ang.dir.numpy())
    print("wrote", a.out)


if __name__ == "__main__":
    main()
