"""The latitude-longitude angle grid (Sec. 2.6) through the C ABI against the
oracle: the grid tables, the step (flat and Kerr-Schild, polar boundaries
through the grid's own pi rotation, angular fluxes over meridian and
latitude sides), the time-step bound, the moments on CUDA and tensor cores,
and one adjoint step.  Tolerances as for the geodesic grid: FP64 1e-12, FP32
2e-5 (steps); moments FP64 1e-13, split-BF16 1e-4 of R^00; CFL 1e-12; VJP
1e-11."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import adjoint as OA
from oracle import cfl as OCFL
from oracle import moments as OM
from oracle import step as OS
from tests.harness import GpuCase, match_bins, oracle_gas, oracle_setup, rel_err, run_both

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nz,npsi", [(1, 4), (4, 8), (9, 18), (20, 40)])
def test_grid_tables_match_oracle(nz, npsi):
    w = W.make("torus3d", n=(4, 4, 2), level=1, latlong=(nz, npsi), with_intensity=False)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        assert gc.n_ang == nz * npsi and gc.n_ap % 4 == 0
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        assert np.abs(gc.dOmega[gmap] - st.ang.dOmega.numpy()).max() < 1e-15
        inv = np.empty_like(gmap)
        inv[gmap] = np.arange(len(gmap))
        for n in range(gc.n_ang):
            nb_g = sorted(int(inv[m]) for m in gc.nbr[gmap[n]] if m >= 0)
            assert nb_g == sorted(st.ang.nbr[n])
    finally:
        gc.close()


LATLONG_CASES = [
    # name, sizes, (n_zeta, n_psi), precision, recon, steps
    ("turb3d", (6, 5, 7), (4, 8), "f64", "plm", 2),          # flat, periodic: no angular flux
    ("torus3d", (6, 6, 4), (4, 8), "f64", "plm", 2),         # Kerr-Schild: polar, outflow, angular fluxes
    ("torus3d", (6, 6, 4), (6, 12), "f32", "plm", 2),
    ("torus3d_big", (6, 4, 4), (3, 6), "f64", "dc", 1),      # moving gas, scattering
    ("torus3d_big", (5, 4, 4), (5, 10), "f32", "plm", 1),
    ("adjoint2d", (10, 8, 1), (5, 10), "f64", "plm", 2),     # 2D Kerr-Schild
    ("turb3d", (5, 4, 6), (9, 18), "f32", "plm", 2),         # 162 bins: the FP32 flat kernel with a fixed row
]


@pytest.mark.parametrize("name,n,ll,prec,recon,steps", LATLONG_CASES)
def test_step_on_latlong_grid_matches_oracle(name, n, ll, prec, recon, steps):
    w = W.make(name, n=n, level=1, latlong=ll)
    r = run_both(w, steps, prec, recon=recon)
    try:
        tol = 1e-12 if prec == "f64" else 2e-5
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
        if prec == "f64":
            assert rel_err(r["src_g"], r["src_o"]) < 1e-11
    finally:
        r["gc"].close()


ANGPLM_CASES = [
    # name, sizes, (n_zeta, n_psi), precision, spatial recon, steps
    ("torus3d", (6, 6, 4), (4, 8), "f64", "plm", 2),         # Kerr-Schild 3D: polar, outflow
    ("torus3d", (6, 6, 4), (6, 12), "f32", "plm", 2),
    ("torus3d_big", (6, 4, 4), (3, 6), "f64", "dc", 1),      # moving gas, scattering
    ("torus3d_big", (5, 4, 4), (5, 10), "f32", "ppm", 1),
    ("adjoint2d", (10, 8, 1), (2, 4), "f64", "plm", 2),      # 2D; two bands: both lines cross a pole
]


@pytest.mark.parametrize("name,n,ll,prec,recon,steps", ANGPLM_CASES)
def test_angular_plm_on_latlong_grid_matches_oracle(name, n, ll, prec, recon, steps):
    """PLM along the lat/long grid lines (continued across the poles) for the
    angular fluxes, against the oracle."""
    w = W.make(name, n=n, level=1, latlong=ll)
    r = run_both(w, steps, prec, recon=recon, recon_ang="plm")
    try:
        tol = 1e-12 if prec == "f64" else 2e-5
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
    finally:
        r["gc"].close()


def test_angular_plm_needs_a_latlong_grid():
    w = W.make("torus3d", n=(4, 4, 2), level=2)
    gc = GpuCase(w)
    try:
        I = torch.zeros((2, 4, 4, gc.n_ap), dtype=torch.float64, device="cuda")
        with pytest.raises(rad.RadError) as e:
            rad.rad_step(gc.ctx, I, gc.gas(w), 0.01, rad.rad_opts_default(recon_ang=rad.RAD_RECON_PLM))
        assert e.value.status == rad.RAD_EUNSUPPORTED
        with pytest.raises(rad.RadError) as e:
            rad.rad_step(gc.ctx, I, gc.gas(w), 0.01, rad.rad_opts_default(recon_ang=5))
        assert e.value.status == rad.RAD_EINVAL
    finally:
        gc.close()
    w = W.make("torus3d", n=(4, 4, 2), level=2)
    gc = GpuCase(w)
    try:
        I = torch.zeros((2, 4, 4, gc.n_ap), dtype=torch.float64, device="cuda")
        z = torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(rad.RadError) as e:        # nor the adjoint on a geodesic grid
            rad.rad_step_adjoint(gc.ctx, I, gc.gas(w), 0.01,
                                 rad.rad_opts_default(coupling=rad.RAD_COUPLE_NONE, recon_ang=rad.RAD_RECON_PLM),
                                 I, torch.zeros_like(I), None, None, z, z.clone())
        assert e.value.status == rad.RAD_EUNSUPPORTED
    finally:
        gc.close()


def test_cfl_on_latlong_grid_matches_oracle():
    w = W.make("torus3d", n=(6, 6, 4), level=1, latlong=(6, 12), with_intensity=False)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        assert abs(rad.rad_cfl_dt(gc.ctx, 0.3) - OCFL.cfl_dt(st, 0.3)) < 1e-12 * OCFL.cfl_dt(st, 0.3)
    finally:
        gc.close()


@pytest.mark.parametrize("method,prec", [(rad.RAD_MOM_SIMT, "f64"), (rad.RAD_MOM_BF16X3, "f32")])
@pytest.mark.parametrize("frame", [rad.RAD_FRAME_TETRAD, rad.RAD_FRAME_FLUID])
def test_moments_on_latlong_grid(method, prec, frame):
    w = W.make("torus3d_big", n=(7, 6, 4), level=1, latlong=(9, 18))
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        tdt = torch.float64 if prec == "f64" else torch.float32
        Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
        R = torch.zeros(Ig.shape[:-1] + (10,), dtype=tdt, device="cuda")
        rad.rad_moments(gc.ctx, Ig, rad.RAD_F64 if prec == "f64" else rad.RAD_F32, frame, method, gc.gas(w), R)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        fr = "tetrad" if frame == rad.RAD_FRAME_TETRAD else "fluid"
        ref = OM.moments(torch.tensor(w["I0"]), st.ang, fr, e=st.e, u=torch.tensor(w["u"])).numpy()
        got = R.double().cpu().numpy()
        if prec == "f64":
            assert rel_err(got, ref) < 1e-13
        else:
            assert (np.abs(got - ref) / np.abs(ref[..., :1])).max() < 1e-4
    finally:
        gc.close()


def test_adjoint_on_latlong_grid_matches_oracle():
    w = W.make("torus3d", n=(6, 6, 4), level=1, latlong=(4, 8))
    rng = np.random.default_rng(17)
    w["eta"] = 10.0 ** rng.uniform(-1, 1, w["T"].shape) / (4 * np.pi)
    w["mode"] = "emissivity"
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        lam = rng.normal(size=w["I0"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, _, ga_o, gs_o, ge_o = OA.step_vjp(I0, T0, oracle_gas(w), dt, st, OS.Opts(mode="emissivity"),
                                                 torch.tensor(lam))
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float64)
        lg = gc.to_gpu_I(lam, gmap, torch.float64)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        ga, gs, ge = (torch.zeros_like(gas["rho"]) for _ in range(3))
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, None, None, ga, gs, ge)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < 1e-11
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 1e-11
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 1e-11
        assert rel_err(ge.cpu().numpy(), ge_o.numpy()) < 1e-11
    finally:
        gc.close()


def test_latlong_arguments_are_checked():
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        for nz, npsi in ((0, 8), (4, 3), (4, 6 + 1), (4, 2), (100, 100)):
            with pytest.raises(rad.RadError) as e:
                rad.rad_init_angles_latlong(ctx, nz, npsi)
            assert e.value.status == rad.RAD_EINVAL
        assert rad.rad_init_angles_latlong(ctx, 2, 4) == (8, 8)
    finally:
        rad.rad_destroy(ctx)


ANGPLM_ADJ_CASES = [
    # name, sizes, (n_zeta, n_psi), spatial recon, coupling, C, precision
    ("torus3d", (6, 6, 4), (4, 8), "plm", "emissivity", 0.0, "f64"),   # Kerr-Schild 3D, polar, outflow
    ("torus3d", (5, 4, 4), (2, 4), "dc", "emissivity", 0.0, "f64"),    # every line crosses a pole
    ("adjoint2d", (10, 8, 1), (5, 10), "plm", "emissivity", 0.0, "f64"),  # 2D
    ("torus3d_big", (5, 4, 4), (3, 6), "plm", "thermal", 0.0, "f64"),  # moving gas, scattering
    ("torus3d", (6, 6, 4), (4, 8), "ppm", "emissivity", 5.0, "f64"),   # with PPM and the optical-depth weighting
    ("torus3d", (6, 6, 4), (6, 12), "plm", "emissivity", 0.0, "f32"),
]


@pytest.mark.parametrize("name,n,ll,recon,coupling,C,prec", ANGPLM_ADJ_CASES)
def test_angular_plm_adjoint_matches_oracle(name, n, ll, recon, coupling, C, prec):
    """The adjoint with PLM angular reconstruction along the lines of the
    lat/long grid (recon_ang) against the oracle's reverse mode: FP64 1e-11
    per output (thermal dL/dalpha_s 2e-10), FP32 2e-4."""
    w = W.make(name, n=n, level=1, latlong=ll)
    rng = np.random.default_rng(19)
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
            I0, T0, oracle_gas(w), dt, st, OS.Opts(recon=recon, mode=coupling, tau_const=C, recon_ang="plm"),
            torch.tensor(lam), None if lamT is None else torch.tensor(lamT))
        f64 = prec == "f64"
        tdt = torch.float64 if f64 else torch.float32
        o = rad.rad_opts_default(precision=rad.RAD_F64 if f64 else rad.RAD_F32,
                                 coupling=rad.RAD_COUPLE_THERMAL if coupling == "thermal" else rad.RAD_COUPLE_EMISSIVITY,
                                 recon={"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM}[recon],
                                 tau_const=C, recon_ang=rad.RAD_RECON_PLM)
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

