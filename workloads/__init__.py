"""Seeded synthetic workloads shaped like the paper's test problems.

This module holds no arithmetic of the radiation method: it only draws
seeded random fields and lays out grids.  It is the one module shared by the
CUDA path (tests, bench) and the oracle.

Five workloads (sizes overridable for scaled-down parity cases):

  hotspot2d   flat space, Cartesian 2D 32x32, periodic, geodesic level 2;
              static gas rho = 1 with a Gaussian hot spot
              T = 1 + 2 exp(-d^2 / (2 * 4^2)), d in cell units; alpha_a = 1,
              alpha_s = 0; I = a T^4 / 4pi (1 + 0.1 U[-1, 1]); 1 step.
  turb3d      flat space, Cartesian 3D 128^3, periodic, level 4; velocity a
              sum of 27 Fourier modes (k in {1,2,3}^3, Gaussian amplitudes,
              uniform phases) rescaled to max |v| = 0.5; alpha_a, alpha_s
              log-uniform on [1e-2, 1e2]; T log-uniform on [0.5, 2]; 10 steps.
  torus3d     Kerr-Schild a = 0.9, 128 x 64 x 64 in (r, theta, phi), r
              log-spaced on [1.5, 50]; level 6; rho = exp(-((r-10)^2 +
              (10 cos theta)^2) / 8) + 1e-4, alpha_a = rho, alpha_s = 0, T = 1,
              u = 0 (normal observers); 5 steps.
  adjoint2d   Kerr-Schild a = 0.5, 256 x 128 in (r, theta), r log on [2, 50];
              level 4; log10 alpha_a, log10 alpha_s, log10(4 pi eta) smooth
              fields in [-1, 1] (3x3 Fourier modes in (log r, theta));
              fixed-emissivity coupling; 8 steps.
  torus3d_big Kerr-Schild a = 0.9, 192 x 96 x 96, level 8, the torus gas
              plus a random velocity (max 0.3, turb3d construction) and
              alpha_s = alpha_a / 2; 20 steps.

Random streams: numpy PCG64 seeded with the workload's seed, drawn in a fixed
order (fields first, then the intensity perturbation).  Intensities are
generated as [n3, n2, n1, n_ang] arrays of perturbation factors in bin-index
order; which direction a bin index means is up to the consumer.
"""
import math

import numpy as np

LEVEL_NANG = {1: 12, 2: 42, 3: 92, 4: 162, 5: 252, 6: 362, 7: 492, 8: 642}


def n_ang(level):
    return 10 * level * level + 2


def _faces_uniform(lo, hi, n):
    return np.linspace(lo, hi, n + 1)


def _faces_log(lo, hi, n):
    return np.exp(np.linspace(math.log(lo), math.log(hi), n + 1))


def _centres(xf):
    return 0.5 * (xf[1:] + xf[:-1])


def _fourier_velocity(rng, xc, vmax):
    """Sum over k in {1,2,3}^3 of a_k sin(2 pi k.x / L + phi_k), per component."""
    X1, X2, X3 = xc
    Z, Y, X = np.meshgrid(X3, X2, X1, indexing="ij")
    L = [X1[-1] - X1[0] + (X1[1] - X1[0] if len(X1) > 1 else 1.0),
         X2[-1] - X2[0] + (X2[1] - X2[0] if len(X2) > 1 else 1.0),
         X3[-1] - X3[0] + (X3[1] - X3[0] if len(X3) > 1 else 1.0)]
    v = np.zeros(Z.shape + (3,))
    for comp in range(3):
        for k1 in (1, 2, 3):
            for k2 in (1, 2, 3):
                for k3 in (1, 2, 3):
                    amp = rng.normal()
                    ph = rng.uniform(0.0, 2.0 * math.pi)
                    v[..., comp] += amp * np.sin(2 * math.pi * (k1 * X / L[0] + k2 * Y / L[1]
                                                                + k3 * Z / L[2]) + ph)
    vm = np.sqrt((v * v).sum(-1)).max()
    v *= vmax / vm
    gam = 1.0 / np.sqrt(1.0 - (v * v).sum(-1))
    return v * gam[..., None]          # u^ihat = gamma v^i


def _smooth_field(rng, xr, xt):
    """Sum of 3x3 Fourier modes in (x, theta), rescaled to [-1, 1]."""
    T, R = np.meshgrid(xt, xr, indexing="ij")
    f = np.zeros_like(R)
    for m in (1, 2, 3):
        for n in (1, 2, 3):
            f += rng.normal() * np.cos(2 * math.pi * m * R + rng.uniform(0, 2 * math.pi)) \
                 * np.cos(2 * n * T)
    f = (f - f.min()) / (f.max() - f.min())
    return 2.0 * f - 1.0


def torus_density(r, th):
    return np.exp(-((r - 10.0) ** 2 + (10.0 * np.cos(th)) ** 2) / 8.0) + 1e-4


def make(name, n=None, level=None, seed=None, with_intensity=True, latlong=None):
    """Return a dict describing one workload (all float64 numpy arrays).

    keys: kind, spin, xf (3 face arrays), bc, ndim, level, nsteps, cfl, mode,
          rho, u [n3,n2,n1,3], alpha_a, alpha_s, eta, T, and (if
          with_intensity) I0 [n3,n2,n1,n_ang].
    """
    w = {"name": name, "cfl": 0.3, "mode": "thermal"}
    if name == "hotspot2d":
        n = n or (32, 32, 1)
        level = level or 2
        seed = 0 if seed is None else seed
        w.update(kind="mink_cart", spin=0.0, ndim=2, nsteps=1,
                 xf=[_faces_uniform(0, 1, n[0]), _faces_uniform(0, 1, n[1]), _faces_uniform(0, 1, 1)],
                 bc=(("periodic", "periodic"), ("periodic", "periodic"), ("periodic", "periodic")))
    elif name == "turb3d":
        n = n or (128, 128, 128)
        level = level or 4
        seed = 1 if seed is None else seed
        w.update(kind="mink_cart", spin=0.0, ndim=3, nsteps=10,
                 xf=[_faces_uniform(0, 1, n[0]), _faces_uniform(0, 1, n[1]), _faces_uniform(0, 1, n[2])],
                 bc=(("periodic", "periodic"),) * 3)
    elif name in ("torus3d", "torus3d_big"):
        big = name == "torus3d_big"
        n = n or ((192, 96, 96) if big else (128, 64, 64))
        level = level or (8 if big else 6)
        seed = (5 if big else 2) if seed is None else seed
        w.update(kind="ks_sph", spin=0.9, ndim=3, nsteps=20 if big else 5,
                 xf=[_faces_log(1.5, 50.0, n[0]), _faces_uniform(0, math.pi, n[1]),
                     _faces_uniform(0, 2 * math.pi, n[2])],
                 bc=(("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")))
    elif name == "adjoint2d":
        n = n or (256, 128, 1)
        level = level or 4
        seed = 3 if seed is None else seed
        w.update(kind="ks_sph", spin=0.5, ndim=2, nsteps=8, mode="emissivity",
                 xf=[_faces_log(2.0, 50.0, n[0]), _faces_uniform(0, math.pi, n[1]),
                     _faces_uniform(0, 2 * math.pi, 1)],
                 bc=(("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")))
    else:
        raise ValueError(name)
    w["level"], w["seed"], w["n"] = level, seed, tuple(n)
    # angle grid: the geodesic grid of the level, or a (n_zeta, n_psi)
    # latitude-longitude grid in its place
    w["latlong"] = tuple(latlong) if latlong is not None else None
    rng = np.random.Generator(np.random.PCG64(seed))
    xc = [_centres(x) for x in w["xf"]]
    shape = (n[2], n[1], n[0])
    Z, Y, X = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    w["eta"] = None
    if name == "hotspot2d":
        w["rho"] = np.ones(shape)
        w["u"] = np.zeros(shape + (3,))
        ci, cj = np.meshgrid(np.arange(n[1]) + 0.5, np.arange(n[0]) + 0.5, indexing="ij")
        d2 = (ci - n[1] / 2.0) ** 2 + (cj - n[0] / 2.0) ** 2
        w["T"] = np.broadcast_to(1.0 + 2.0 * np.exp(-d2 / (2.0 * 16.0)), shape).copy()
        w["alpha_a"] = np.ones(shape)
        w["alpha_s"] = np.zeros(shape)
    elif name == "turb3d":
        w["rho"] = np.ones(shape)
        w["u"] = _fourier_velocity(rng, xc, 0.5)
        w["alpha_a"] = 10.0 ** rng.uniform(-2, 2, shape)
        w["alpha_s"] = 10.0 ** rng.uniform(-2, 2, shape)
        w["T"] = np.exp(rng.uniform(math.log(0.5), math.log(2.0), shape))
    elif name in ("torus3d", "torus3d_big"):
        rho = torus_density(X, Y)
        w["rho"] = rho
        w["alpha_a"] = rho.copy()
        w["T"] = np.ones(shape)
        if name == "torus3d_big":
            w["u"] = _fourier_velocity(rng, xc, 0.3)
            w["alpha_s"] = 0.5 * rho
        else:
            w["u"] = np.zeros(shape + (3,))
            w["alpha_s"] = np.zeros(shape)
    elif name == "adjoint2d":
        lr = (np.log(xc[0]) - math.log(2.0)) / (math.log(50.0) - math.log(2.0))
        fa = _smooth_field(rng, lr, xc[1])
        fs = _smooth_field(rng, lr, xc[1])
        fe = _smooth_field(rng, lr, xc[1])
        w["rho"] = np.ones(shape)
        w["u"] = np.zeros(shape + (3,))
        w["T"] = np.ones(shape)
        w["alpha_a"] = (10.0 ** fa)[None].copy()
        w["alpha_s"] = (10.0 ** fs)[None].copy()
        w["eta"] = ((10.0 ** fe) / (4 * math.pi))[None].copy()
    # position of the generator where the intensity draws start (intensity_rows
    # draws any rows of I0 from here without forming the whole array)
    w["_rng_I0"] = rng.bit_generator.state
    w["n_ang"] = n_ang(level) if latlong is None else latlong[0] * latlong[1]
    if with_intensity:
        na = w["n_ang"]
        U = rng.uniform(-1.0, 1.0, shape + (na,))
        if name == "adjoint2d":
            base = np.full(shape, 1.0 / (4 * math.pi))
        else:
            base = w["T"] ** 4 / (4 * math.pi)
        w["I0"] = base[..., None] * (1.0 + 0.1 * U)
    return w


def _base_intensity(w, k, j):
    """a_rad T^4 / 4 pi (1 / 4 pi for adjoint2d) of the x1 row (k, j)."""
    if w["name"] == "adjoint2d":
        return np.full(w["n"][0], 1.0 / (4 * math.pi))
    return w["T"][k, j] ** 4 / (4 * math.pi)


def intensity_rows(w, k, j=None):
    """Rows of the initial intensity I0 without forming the whole array: the
    x1 row (k, j) as [n1, n_ang], or with j None the whole x3 slab k as
    [n2, n1, n_ang].  Equal to make(...)["I0"][k, j] / ["I0"][k]: every
    uniform draw takes one 64-bit output of PCG64, so the generator is
    advanced to the row's first element."""
    n1, n2, _ = w["n"]
    na = w["n_ang"]
    bg = np.random.PCG64()
    bg.state = w["_rng_I0"]
    if j is None:
        bg.advance(k * n2 * n1 * na)
        U = np.random.Generator(bg).uniform(-1.0, 1.0, (n2, n1, na))
        base = np.stack([_base_intensity(w, k, jj) for jj in range(n2)])
        return base[..., None] * (1.0 + 0.1 * U)
    bg.advance((k * n2 + j) * n1 * na)
    U = np.random.Generator(bg).uniform(-1.0, 1.0, (n1, na))
    return _base_intensity(w, k, j)[:, None] * (1.0 + 0.1 * U)


def fd_cells(w, count=16):
    """Cells (k, j, i) drawn with the workload seed for finite-difference checks."""
    rng = np.random.Generator(np.random.PCG64(w["seed"] + 1000))
    n = w["n"]
    flat = rng.choice(n[0] * n[1] * n[2], size=count, replace=False)
    return [(int(f // (n[0] * n[1])), int((f // n[0]) % n[1]), int(f % n[0])) for f in flat]
