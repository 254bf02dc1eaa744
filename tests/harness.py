"""Test harness: runs one workload through the CUDA library (via the Python
binding) and through the oracle, on the same seeded inputs, and maps the two
angle orderings onto each other by matching directions."""
import math

import numpy as np
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import cfl as OCFL
from oracle import step as OS
from oracle.angles import GeodesicGrid, LatLongGrid
from oracle.transport import Grid, Setup

_SETUPS = {}


def oracle_setup(w):
    key = (w["name"], w["n"], w["level"], w["kind"], w["spin"], w.get("latlong"))
    if key not in _SETUPS:
        ang = GeodesicGrid(w["level"]) if w.get("latlong") is None else LatLongGrid(*w["latlong"])
        _SETUPS[key] = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), ang)
    return _SETUPS[key]


def match_bins(gpu_dir, ora_dir):
    """g[n] = GPU bin of oracle bin n; asserts a bijection with error < 1e-13."""
    d2 = ((ora_dir[:, None, :] - gpu_dir[None, :, :]) ** 2).sum(-1)
    g = d2.argmin(axis=1)
    assert sorted(g.tolist()) == list(range(len(g)))
    assert float(np.sqrt(d2[np.arange(len(g)), g].max())) < 1e-13
    return g


class GpuCase:
    """Library context set up for workload w (same grid and angle level)."""

    def __init__(self, w, dev="cuda:0"):
        self.w = w
        self.dev = dev
        self.stream = torch.cuda.current_stream()
        self.ctx = rad.rad_create(self.stream)
        if w.get("latlong") is None:
            self.n_ang, self.n_ap = rad.rad_init_angles(self.ctx, w["level"])
        else:
            self.n_ang, self.n_ap = rad.rad_init_angles_latlong(self.ctx, *w["latlong"])
        self.dir, self.dOmega, self.nbr = rad.rad_get_angles(self.ctx, self.n_ang)
        rad.rad_set_metric(self.ctx, w["kind"], w["spin"], w["ndim"], w["xf"], w["bc"])

    def close(self):
        torch.cuda.synchronize()
        rad.rad_destroy(self.ctx)

    def to_gpu_I(self, I_ora, gmap, dtype):
        """Oracle-ordered [.., n_ang] -> padded GPU layout [.., n_ap] on the device."""
        sh = I_ora.shape[:-1]
        out = np.zeros(sh + (self.n_ap,))
        out[..., gmap] = I_ora
        return torch.tensor(out, dtype=dtype, device=self.dev).contiguous()

    def from_gpu_I(self, I_gpu, gmap):
        return I_gpu.double().cpu().numpy()[..., gmap]

    def gas(self, w, T=None):
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=self.dev)
        g = {"rho": t(w["rho"]), "u": t(w["u"]), "alpha_a": t(w["alpha_a"]), "alpha_s": t(w["alpha_s"]),
             "eta": t(w["eta"]) if w["eta"] is not None else None,
             "T": t(w["T"] if T is None else T)}
        return g


def oracle_gas(w):
    g = {k: torch.tensor(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s")}
    g["eta"] = torch.tensor(w["eta"]) if w["eta"] is not None else None
    return g


def run_both(w, nsteps, precision="f64", recon="plm", coupling=None, dt=None, tau=0.0, rad_dom=False,
             recon_ang="dc"):
    """Advance workload w nsteps on the GPU and in the oracle; return both states."""
    st = oracle_setup(w)
    gc = GpuCase(w)
    gmap = match_bins(gc.dir, st.ang.dir.numpy())
    mode = coupling or w["mode"]
    if dt is None:
        dt = OCFL.cfl_dt(st, w["cfl"])
    # oracle
    opts = OS.Opts(recon=recon, mode=mode if mode != "none" else "thermal", couple=mode != "none",
                   tau_const=tau, rad_dom=rad_dom, recon_ang=recon_ang)
    I, T = torch.tensor(w["I0"]), torch.tensor(w["T"])
    gas_o = oracle_gas(w)
    src_tot = torch.zeros(T.shape + (4,), dtype=torch.float64)
    for _ in range(nsteps):
        I, T, src, ok = OS.rk2_step(I, T, gas_o, dt, st, opts)
        assert bool(ok.all())
        src_tot = src
    # GPU
    tdt = torch.float64 if precision == "f64" else torch.float32
    Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
    gas_g = gc.gas(w)
    src_g = torch.zeros(T.shape + (4,), dtype=torch.float64, device=gc.dev)
    cmode = {"thermal": rad.RAD_COUPLE_THERMAL, "emissivity": rad.RAD_COUPLE_EMISSIVITY,
             "none": rad.RAD_COUPLE_NONE}[mode]
    o = rad.rad_opts_default(precision=rad.RAD_F64 if precision == "f64" else rad.RAD_F32,
                             recon={"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM}[recon],
                             coupling=cmode, tau_const=tau, rad_dom=int(rad_dom),
                             recon_ang={"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM,
                                        "mapr": rad.RAD_RECON_MAPR}[recon_ang])
    for _ in range(nsteps):
        rad.rad_step(gc.ctx, Ig, gas_g, dt, o, src_g)
    rad.rad_check(gc.ctx)
    torch.cuda.synchronize()
    out = {"I_o": I.numpy(), "T_o": T.numpy(), "src_o": src_tot.numpy(),
           "I_g": gc.from_gpu_I(Ig, gmap), "T_g": gas_g["T"].cpu().numpy(), "src_g": src_g.cpu().numpy(),
           "I_g_raw": Ig, "gmap": gmap, "dt": dt, "gc": gc, "setup": st}
    return out


def rel_err(a, b):
    """max |a - b| / max |b| (normwise relative error)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_err_elem(a, b):
    """max |a - b| / |b| over elements with b != 0 (per-element relative
    error; where b == 0 the two must agree exactly, else inf)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nz = b != 0
    if np.any(a[~nz] != 0):
        return float("inf")
    return float((np.abs(a[nz] - b[nz]) / np.abs(b[nz])).max()) if nz.any() else 0.0
