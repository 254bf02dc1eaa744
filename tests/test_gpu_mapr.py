"""Minimum-angle plane reconstruction (MAPR) of the angular face values on
geodesic grids (recon_ang = RAD_RECON_MAPR) through the C ABI, against the
oracle: FP64 1e-12, FP32 2e-5 relative (normwise per output), as for every
step; the adjoint with it against the oracle's reverse mode (FP64 1e-11,
FP32 2e-4); and the options that refuse it."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import adjoint as OA
from oracle import cfl as OCFL
from oracle import step as OS
from tests.harness import GpuCase, match_bins, oracle_gas, oracle_setup, rel_err, run_both

pytestmark = pytest.mark.gpu

MAPR_CASES = [
    # name, sizes, level, precision, spatial recon, steps
    ("torus3d", (8, 6, 4), 2, "f64", "plm", 2),        # Kerr-Schild 3D, polar, outflow
    ("torus3d", (6, 6, 4), 3, "f64", "dc", 1),         # 92 bins
    ("torus3d_big", (6, 4, 4), 2, "f64", "plm", 1),    # moving gas, scattering
    ("torus3d_big", (5, 4, 4), 1, "f64", "plm", 2),    # level 1: every cell a pentagon
    ("adjoint2d", (10, 8, 1), 2, "f64", "plm", 2),     # 2D, fixed emissivity
    ("torus3d", (8, 6, 4), 2, "f32", "plm", 2),
    ("torus3d", (6, 6, 4), 4, "f32", "ppm", 1),        # 162 bins, PPM in space
]


@pytest.mark.parametrize("name,n,level,prec,recon,steps", MAPR_CASES)
def test_mapr_step_matches_oracle(name, n, level, prec, recon, steps):
    w = W.make(name, n=n, level=level)
    r = run_both(w, steps, prec, recon=recon, recon_ang="mapr")
    try:
        tol = 1e-12 if prec == "f64" else 2e-5
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
        pad = r["I_g_raw"][..., r["gc"].n_ang:]
        assert pad.abs().max().item() == 0.0 if pad.numel() else True
    finally:
        r["gc"].close()


def test_mapr_differs_from_donor_cell():
    """The reconstruction acts: one step with MAPR and one with DC angular
    fluxes differ by far more than the parity tolerance."""
    w = W.make("torus3d", n=(8, 6, 4), level=2)
    a = run_both(w, 1, "f64", recon_ang="mapr")
    b = run_both(w, 1, "f64", recon_ang="dc")
    try:
        assert rel_err(a["I_g"], b["I_g"]) > 1e-6
    finally:
        a["gc"].close()
        b["gc"].close()


def test_mapr_arguments_are_checked():
    w = W.make("torus3d", n=(4, 4, 2), level=1, latlong=(2, 4))
    gc = GpuCase(w)
    try:
        I = torch.zeros((2, 4, 4, gc.n_ap), dtype=torch.float64, device="cuda")
        with pytest.raises(rad.RadError) as e:           # MAPR needs a geodesic grid
            rad.rad_step(gc.ctx, I, gc.gas(w), 0.01, rad.rad_opts_default(recon_ang=rad.RAD_RECON_MAPR))
        assert e.value.status == rad.RAD_EUNSUPPORTED
    finally:
        gc.close()
    w = W.make("torus3d", n=(4, 4, 2), level=2)
    gc = GpuCase(w)
    try:
        I = torch.zeros((2, 4, 4, gc.n_ap), dtype=torch.float64, device="cuda")
        z = torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(rad.RadError) as e:           # as a spatial reconstruction it is unknown
            rad.rad_step(gc.ctx, I, gc.gas(w), 0.01, rad.rad_opts_default(recon=rad.RAD_RECON_MAPR))
        assert e.value.status == rad.RAD_EINVAL
    finally:
        gc.close()


MAPR_ADJ_CASES = [
    # name, sizes, level, spatial recon, coupling, C, precision
    ("torus3d", (6, 6, 4), 2, "plm", "emissivity", 0.0, "f64"),
    ("torus3d_big", (5, 4, 4), 1, "plm", "thermal", 0.0, "f64"),      # pentagons, moving gas, scattering
    ("adjoint2d", (10, 8, 1), 2, "ppm", "emissivity", 5.0, "f64"),    # 2D, PPM, optical-depth weighting
    ("torus3d", (6, 6, 4), 2, "plm", "emissivity", 0.0, "f32"),
]


@pytest.mark.parametrize("name,n,level,recon,coupling,C,prec", MAPR_ADJ_CASES)
def test_mapr_adjoint_matches_oracle(name, n, level, recon, coupling, C, prec):
    w = W.make(name, n=n, level=level)
    rng = np.random.default_rng(23)
    if coupling == "emissivity":
        if w["eta"] is None:
            w["eta"] = 10.0 ** rng.uniform(-1, 1, w["T"].shape) / (4 * np.pi)
    else:
        w["eta"] = None
    w["mode"] = coupling
    if C > 0 and not np.any(w["u"]):
        v = rng.uniform(-1, 1, w["u"].shape)
        v *= 0.3 / np.sqrt((v * v).sum(-1)).max()
        w["u"] = v / np.sqrt(1 - (v * v).sum(-1))[..., None]
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        lam = rng.normal(size=w["I0"].shape)
        lamT = rng.normal(size=w["T"].shape) if coupling == "thermal" else None
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, lamT_o, ga_o, gs_o, ge_o = OA.step_vjp(
            I0, T0, oracle_gas(w), dt, st, OS.Opts(recon=recon, mode=coupling, tau_const=C, recon_ang="mapr"),
            torch.tensor(lam), None if lamT is None else torch.tensor(lamT))
        f64 = prec == "f64"
        tdt = torch.float64 if f64 else torch.float32
        o = rad.rad_opts_default(precision=rad.RAD_F64 if f64 else rad.RAD_F32,
                                 coupling=rad.RAD_COUPLE_THERMAL if coupling == "thermal" else rad.RAD_COUPLE_EMISSIVITY,
                                 recon={"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM}[recon],
                                 tau_const=C, recon_ang=rad.RAD_RECON_MAPR)
        Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
        lg = gc.to_gpu_I(lam, gmap, tdt)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        lTg = None if lamT is None else torch.tensor(lamT, device="cuda")
        lTn = None if lamT is None else torch.zeros_like(lTg)
        ga, gs = torch.zeros_like(gas["rho"]), torch.zeros_like(gas["rho"])
        ge = torch.zeros_like(ga) if coupling == "emissivity" else None
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, lTg, lTn, ga, gs, ge)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        tol = 1e-11 if f64 else 2e-4
        assert rel_err(gc.from_gpu_I(ln.double(), gmap), lam_o.numpy()) < tol
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < tol
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < (2e-10 if f64 and coupling == "thermal" else tol)
        if ge is not None:
            assert rel_err(ge.cpu().numpy(), ge_o.numpy()) < tol
        if lTn is not None:
            assert rel_err(lTn.cpu().numpy(), lamT_o.numpy()) < tol
    finally:
        gc.close()

