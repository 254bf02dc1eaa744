"""Expected values of a benchmark workload advanced over its stated number of
RK2 steps on its full grid, at seeded sample points, written by the FP64
oracle alone (test infrastructure; nothing here comes from the CUDA path).

  turb3d   flat Cartesian 128^3, geodesic level 4 (162 bins), periodic,
           moving gas |v| <= 0.5, log-uniform opacities and temperatures,
           thermal coupling, PLM: 10 steps
  torus3d  Kerr-Schild a = 0.9, 128 x 64 x 64 (r log on [1.5, 50], full
           theta and phi), level 6 (362 bins), torus gas at rest, thermal
           coupling, PLM: 5 steps

Every step runs on the whole grid, one slab at a time to bound the memory:
a slab's cells are advanced from a window that reaches four cells beyond it
(two RK stages of a stencil that reaches two cells), so the slab's results
are those of the whole-grid step.  turb3d is cut along x3 (periodic; the
geometry does not depend on x3, so one window geometry serves every slab);
torus3d along x1 (its polar boundary pairs phi with phi + pi, so x3 stays
whole).  dt = 0.3 x the oracle's time-step bound.

Samples (numpy PCG64, seed 30): 4096 cells, for torus3d including every
cell within four of the radial and polar boundaries in a few columns, with
T, the gas source of the last step and the tetrad-frame moments R there;
8192 (cell, bin) intensities (oracle bin order) and the oracle grid's bin
directions (to pair its bins with another grid's).

    python tests/golden/make_config_samples.py turb3d|torus3d

writes tests/golden/<name>_samples.npz.
"""
import argparse
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

M = 4            # window reach beyond a slab: two stages x two cells
NCELL = 4096
NBIN = 8192


def step_slabs_x3(w, ang, I, T, gas, dt, slab):
    """One step of a grid periodic in x3, slab by slab along x3."""
    n3 = I.shape[0]
    dphi = float(w["xf"][2][1] - w["xf"][2][0])
    xf = [w["xf"][0], w["xf"][1], dphi * np.arange(slab + 2 * M + 1)]
    st = Setup(Grid(w["kind"], w["spin"], xf, (w["bc"][0], w["bc"][1], ("outflow", "outflow")), 3), ang)
    I2, T2, src = torch.empty_like(I), torch.empty_like(T), torch.empty(T.shape + (4,), dtype=T.dtype)
    for k0 in range(0, n3, slab):
        kk = torch.tensor(np.arange(k0 - M, k0 + slab + M) % n3)
        g = {k: v[kk] for k, v in gas.items() if v is not None}
        g["eta"] = None
        a, b, c, ok = OS.rk2_step(I[kk], T[kk], g, dt, st, OS.Opts())
        assert bool(ok.all())
        I2[k0:k0 + slab], T2[k0:k0 + slab], src[k0:k0 + slab] = a[M:M + slab], b[M:M + slab], c[M:M + slab]
    return I2, T2, src


def step_slabs_x1(w, ang, I, T, gas, dt, slab, setups):
    """One step of a grid with outflow x1 boundaries, slab by slab along x1."""
    n1 = I.shape[2]
    I2, T2, src = torch.empty_like(I), torch.empty_like(T), torch.empty(T.shape + (4,), dtype=T.dtype)
    for i0 in range(0, n1, slab):
        lo, hi = max(0, i0 - M), min(n1, i0 + slab + M)
        st = setups.get(i0) if setups is not None else None
        if st is None:
            bc = ("outflow", "outflow")     # the true boundary where the window reaches it, a cut elsewhere
            xf = [w["xf"][0][lo:hi + 1], w["xf"][1], w["xf"][2]]
            st = Setup(Grid(w["kind"], w["spin"], xf, (bc, w["bc"][1], w["bc"][2]), 3), ang)
            if setups is not None:
                setups[i0] = st
        g = {k: v[:, :, lo:hi].contiguous() for k, v in gas.items() if v is not None}
        g["eta"] = None
        a, b, c, ok = OS.rk2_step(I[:, :, lo:hi].contiguous(), T[:, :, lo:hi].contiguous(), g, dt, st, OS.Opts())
        del st
        assert bool(ok.all())
        s = slice(i0 - lo, i0 - lo + min(slab, n1 - i0))
        I2[:, :, i0:i0 + slab], T2[:, :, i0:i0 + slab], src[:, :, i0:i0 + slab] = a[:, :, s], b[:, :, s], c[:, :, s]
    return I2, T2, src


def sample_cells(w, rng):
    n1, n2, n3 = w["n"]
    cells = np.stack([rng.integers(0, n3, NCELL), rng.integers(0, n2, NCELL), rng.integers(0, n1, NCELL)], 1)
    if w["kind"] != "mink_cart":
        # every cell within four of the radial and polar boundaries in four (k, j) / (k, i) lines
        extra = []
        for k in rng.integers(0, n3, 2):
            for i in list(range(4)) + list(range(n1 - 4, n1)):
                for j in rng.integers(0, n2, 2):
                    extra.append((k, j, i))
            for j in list(range(4)) + list(range(n2 - 4, n2)):
                for i in rng.integers(0, n1, 2):
                    extra.append((k, j, i))
        cells[:len(extra)] = np.array(extra)
    return cells


def main():
    p = argparse.ArgumentParser()
    p.add_argument("name", choices=["turb3d", "torus3d"])
    p.add_argument("--add-dirs", action="store_true", help="only add the bin directions to an existing file")
    a = p.parse_args()
    w = W.make(a.name, with_intensity=False)
    if a.add_dirs:
        add_dirs(os.path.join(HERE, f"{a.name}_samples.npz"), w["level"])
        return
    ang = GeodesicGrid(w["level"])
    n1, n2, n3 = w["n"]
    if a.name == "turb3d":
        dt = OCFL.cfl_dt(Setup(Grid(w["kind"], w["spin"], [w["xf"][0], w["xf"][1], w["xf"][2][:2]],
                                    (w["bc"][0], w["bc"][1], ("periodic", "periodic")), 3), ang), w["cfl"])
    else:
        xf1 = [w["xf"][0], w["xf"][1], w["xf"][2][:2]]
        dt = OCFL.cfl_dt(Setup(Grid(w["kind"], w["spin"], xf1, (w["bc"][0], w["bc"][1], ("periodic", "periodic")), 3),
                               ang), w["cfl"])
    print("dt", dt, flush=True)
    I = torch.tensor(np.stack([W.intensity_rows(w, k) for k in range(n3)]))
    T = torch.tensor(w["T"])
    gas = {k: torch.tensor(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s")}
    gas["eta"] = None
    for s in range(w["nsteps"]):
        t0 = time.time()
        if a.name == "turb3d":
            I, T, src = step_slabs_x3(w, ang, I, T, gas, dt, 16)
        else:
            I, T, src = step_slabs_x1(w, ang, I, T, gas, dt, 32, None)   # geometry rebuilt per slab (memory)
        print(f"step {s + 1}/{w['nsteps']} {time.time() - t0:.0f} s", flush=True)
    rng = np.random.default_rng(30)
    cells = sample_cells(w, rng)
    kc, jc, ic = cells[:, 0], cells[:, 1], cells[:, 2]
    R = OM.moments(I[kc, jc, ic], ang).numpy()
    bcells = np.stack([rng.integers(0, n3, NBIN), rng.integers(0, n2, NBIN), rng.integers(0, n1, NBIN)], 1)
    bins = rng.integers(0, ang.n_ang, NBIN)
    vals = I[bcells[:, 0], bcells[:, 1], bcells[:, 2], bins].numpy()
    out = os.path.join(HERE, f"{a.name}_samples.npz")
    np.savez_compressed(out, cells=cells, T=T[kc, jc, ic].numpy(), src=src[kc, jc, ic].numpy(), R=R,
                        bin_cells=bcells, bins=bins, I=vals, dt=dt, steps=w["nsteps"], dirs=ang.dir.numpy())
    print("wrote", out)


def add_dirs(path, level):
    """Store the oracle grid's bin directions beside values written before
    they were stored (they pair the oracle's bins with another grid's)."""
    d = dict(np.load(path))
    d["dirs"] = GeodesicGrid(level).dir.numpy()
    np.savez_compressed(path, **d)


if __name__ == "__main__":
    main()
