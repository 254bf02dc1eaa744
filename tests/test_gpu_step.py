"""Parity of the CUDA step (rad_step through the C ABI) with the oracle.

Tolerances: FP64 path 1e-12 relative (normwise, max |gpu - oracle| /
max |oracle| per output array); FP32 path 2e-5 relative for I after the
listed steps (FP32 transport and coupling sums, FP64 quartic).  Per element
(max |gpu - oracle| / |oracle|, guarded zeros equal exactly) the intensity
also holds to 1e-10 (FP64) and 2e-3 (FP32): a dim cell's flux difference
carries the rounding of its bright neighbours, so the per-element bound is
the normwise one times the dynamic range of the inputs (256 in turb3d)."""
import math

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from tests.harness import GpuCase, match_bins, rel_err, rel_err_elem, run_both

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

CASES = [
    # name, sizes (n1, n2, n3), level, steps
    ("hotspot2d", (32, 32, 1), 2, 1),
    ("hotspot2d", (13, 7, 1), 1, 2),              # ragged, level 1 (12 bins)
    ("turb3d", (9, 6, 7), 2, 2),                  # odd sizes: ragged batches along x3
    ("turb3d", (6, 5, 12), 4, 1),                 # 162 bins
    ("torus3d", (8, 6, 4), 2, 2),                 # Kerr-Schild: angular fluxes, polar, outflow
    ("torus3d", (6, 8, 6), 3, 1),                 # 92 bins
    ("torus3d_big", (6, 4, 4), 2, 2),             # moving gas + scattering in Kerr-Schild
    ("adjoint2d", (10, 8, 1), 2, 2),              # 2D Kerr-Schild, fixed emissivity
    ("turb3d", (4, 3, 37), 2, 1),                 # x3 longer than one 32-cell chunk, ragged tail
    ("torus3d_big", (3, 4, 10), 8, 1),            # 642 bins: FP64 ring two stages deep
    ("turb3d", (5, 4, 45), 4, 1),                 # the level-4 fixed-row kernel: chunks of 32 + 13 cells
    ("turb3d", (4, 4, 38), 4, 2),                 # ... and 32 + 6 (phase C in eights, fours, pairs, ones)
]


@pytest.mark.parametrize("name,n,level,steps", CASES)
def test_step_f64_matches_oracle(name, n, level, steps):
    w = W.make(name, n=n, level=level)
    r = run_both(w, steps, "f64")
    try:
        assert rel_err(r["I_g"], r["I_o"]) < TOL64
        assert rel_err_elem(r["I_g"], r["I_o"]) < 1e-10
        assert rel_err(r["T_g"], r["T_o"]) < TOL64
        assert rel_err_elem(r["T_g"], r["T_o"]) < 1e-11
        if w["mode"] == "thermal":
            assert rel_err(r["src_g"], r["src_o"]) < 1e-11
        # padding bins are never written
        pad = r["I_g_raw"][..., r["gc"].n_ang:]
        assert pad.abs().max().item() == 0.0 if pad.numel() else True
    finally:
        r["gc"].close()


@pytest.mark.parametrize("name,n,level,steps", [CASES[0], CASES[2], CASES[4], CASES[6], CASES[8], CASES[9],
                                                 CASES[10], CASES[11]])
def test_step_f32_matches_oracle(name, n, level, steps):
    w = W.make(name, n=n, level=level)
    r = run_both(w, steps, "f32")
    try:
        assert rel_err(r["I_g"], r["I_o"]) < TOL32
        assert rel_err_elem(r["I_g"], r["I_o"]) < 2e-3
        assert rel_err(r["T_g"], r["T_o"]) < TOL32
        assert rel_err_elem(r["T_g"], r["T_o"]) < 2e-4
    finally:
        r["gc"].close()


@pytest.mark.parametrize("recon", ["dc", "plm"])
def test_transport_only_f64(recon):
    w = W.make("torus3d", n=(7, 6, 4), level=2)
    r = run_both(w, 2, "f64", recon=recon, coupling="none")
    try:
        assert rel_err(r["I_g"], r["I_o"]) < TOL64
    finally:
        r["gc"].close()


def test_uniform_equilibrium_is_fixed_point_on_gpu():
    w = W.make("turb3d", n=(6, 6, 6), level=2)
    w["I0"] = np.broadcast_to((w["T"] ** 4 / (4 * math.pi))[..., None], w["I0"].shape).copy()
    w["T"] = np.full_like(w["T"], 1.3)
    w["I0"] = np.full_like(w["I0"], 1.3 ** 4 / (4 * math.pi))
    w["u"] = np.zeros_like(w["u"])
    r = run_both(w, 1, "f64")
    try:
        assert np.abs(r["I_g"] - w["I0"]).max() < 1e-15
        assert np.abs(r["T_g"] - 1.3).max() < 1e-14
    finally:
        r["gc"].close()


def test_largest_level_step_f64():
    """Geodesic level 9 (812 bins, the largest rad_step accepts: 416 consumer
    threads and the producer warp): the FP64 stencil ring is two stages deep."""
    w = W.make("torus3d", n=(3, 4, 4), level=9)
    r = run_both(w, 1, "f64")
    try:
        assert rel_err(r["I_g"], r["I_o"]) < TOL64
        assert rel_err(r["T_g"], r["T_o"]) < TOL64
    finally:
        r["gc"].close()


GEO4_F32_CASES = [
    # sizes, recon, C (optical depth): the FP32 flat kernels with the row length
    # of the level-4 geodesic grid (162 bins, 164 padded) fixed at compile time
    ((6, 5, 12), "dc", 0.0),
    ((6, 5, 12), "plm", 0.0),
    ((7, 5, 9), "ppm", 0.0),
    ((5, 4, 35), "plm", 3.0),          # two x3 chunks, ragged tail
    ((7, 5, 6), "dc", 3.0),
    ((7, 5, 6), "ppm", 3.0),
]


@pytest.mark.parametrize("n,recon,C", GEO4_F32_CASES)
def test_step_f32_level4_specialised_matches_oracle(n, recon, C):
    """Both stages of the specialised 164-wide FP32 kernels against the oracle
    (2e-5, as for every FP32 step)."""
    w = W.make("turb3d", n=n, level=4)
    r = run_both(w, 2, "f32", recon=recon, tau=C)
    try:
        assert r["gc"].n_ang == 162
        assert rel_err(r["I_g"], r["I_o"]) < TOL32
        assert rel_err(r["T_g"], r["T_o"]) < TOL32
        pad = r["I_g_raw"][..., r["gc"].n_ang:]
        assert pad.abs().max().item() == 0.0
    finally:
        r["gc"].close()


GEOFIX_ANG_F32_CASES = [
    # name, sizes, level, recon, C, steps: the FP32 curved-space kernels with
    # the row length of the level-4, 6 and 8 geodesic grids fixed at compile time
    ("torus3d", (6, 5, 4), 4, "plm", 0.0, 2),
    ("torus3d", (6, 5, 4), 4, "dc", 0.0, 1),
    ("torus3d", (5, 4, 4), 6, "plm", 0.0, 1),
    ("torus3d", (5, 4, 4), 6, "ppm", 0.0, 1),
    ("torus3d_big", (3, 4, 6), 8, "plm", 0.0, 1),
    ("torus3d_big", (4, 4, 4), 4, "plm", 20.0, 1),     # optical-depth weighting, moving gas
    ("adjoint2d", (10, 8, 1), 4, "plm", 0.0, 2),        # 2D, fixed emissivity
]


@pytest.mark.parametrize("name,n,level,recon,C,steps", GEOFIX_ANG_F32_CASES)
def test_step_f32_curved_fixed_row_matches_oracle(name, n, level, recon, C, steps):
    w = W.make(name, n=n, level=level)
    r = run_both(w, steps, "f32", recon=recon, tau=C)
    try:
        assert r["gc"].n_ang == 10 * level ** 2 + 2
        assert rel_err(r["I_g"], r["I_o"]) < TOL32
        assert rel_err(r["T_g"], r["T_o"]) < TOL32
        pad = r["I_g_raw"][..., r["gc"].n_ang:]
        assert pad.abs().max().item() == 0.0
    finally:
        r["gc"].close()


TAU_CASES = [
    # name, sizes, level, precision, recon, C
    ("turb3d", (7, 5, 6), 2, "f64", "plm", 3.0),       # flat, periodic, moving gas
    ("turb3d", (7, 5, 6), 2, "f32", "plm", 3.0),
    ("turb3d", (5, 4, 35), 2, "f64", "dc", 10.0),      # two x3 chunks
    ("torus3d_big", (6, 6, 4), 2, "f64", "plm", 50.0),  # Kerr-Schild, polar, outflow, moving gas
    ("adjoint2d", (9, 8, 1), 2, "f64", "plm", 5.0),     # 2D (given a moving gas below)
]


@pytest.mark.parametrize("name,n,level,prec,recon,C", TAU_CASES)
def test_optical_depth_weighted_flux_matches_oracle(name, n, level, prec, recon, C):
    """The optical-depth weighting of the spatial fluxes (Sec. 2.4) against
    the oracle; FP64 1e-12, FP32 2e-5 as for the free-streaming step."""
    w = W.make(name, n=n, level=level)
    if not np.any(w["u"]):       # the weighting acts only across velocity differences
        rng = np.random.default_rng(8)
        v = rng.uniform(-1, 1, w["u"].shape)
        v *= 0.3 / np.sqrt((v * v).sum(-1)).max()
        w["u"] = v / np.sqrt(1 - (v * v).sum(-1))[..., None]
    r = run_both(w, 1, prec, recon=recon, tau=C)
    try:
        tol = TOL64 if prec == "f64" else TOL32
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
    finally:
        r["gc"].close()


def test_moving_equilibration_trajectory_f64():
    """The moving equilibration of Sec. 3 (u^1 = 1 initially, gas advanced by
    the returned source): 25 GPU steps follow the oracle's trajectory to
    1e-11 (the oracle's agreement with the paper's ODE is pinned on CPU)."""
    from tests.test_oracle_coupling import _gas_from_conserved, _golden
    import oracle.step as OSS
    g = _golden("static_equilibration.txt")
    gam, rho0, aa, p0, E0 = g["gamma"][0], g["rho"][0], g["alpha_a"][0], g["p_gas0"][0], g["u_rad0"][0]
    w = W.make("turb3d", n=(2, 2, 2), level=2)
    w.update(rho=np.full(w["T"].shape, rho0), alpha_a=np.full(w["T"].shape, aa), alpha_s=np.zeros(w["T"].shape))
    from tests.harness import oracle_setup
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        sh = w["T"].shape
        dO = st.ang.dOmega.numpy()
        u00 = math.sqrt(2.0)
        D = rho0 * u00
        wgas = rho0 + gam / (gam - 1) * p0
        state = {"o": [wgas * 2.0 - p0, wgas * u00, rho0, p0, 1.0], "g": [wgas * 2.0 - p0, wgas * u00, rho0, p0, 1.0]}
        I_o = torch.full(sh + (len(dO),), E0 / (4 * math.pi), dtype=torch.float64)
        I_g = gc.to_gpu_I(I_o.numpy(), gmap, torch.float64)
        dt = 0.4
        for s in range(25):
            Eg, Sx, rho, p, u1 = state["o"]
            gas = {"rho": torch.full(sh, rho, dtype=torch.float64), "alpha_a": torch.full(sh, aa, dtype=torch.float64),
                   "alpha_s": torch.zeros(sh, dtype=torch.float64), "eta": None,
                   "u": torch.tensor([u1, 0.0, 0.0], dtype=torch.float64).expand(sh + (3,)).clone()}
            I_o, _, src_o, ok = OSS.rk2_step(I_o, torch.full(sh, p / rho, dtype=torch.float64), gas, dt, st,
                                             OSS.Opts(recon="dc", gamma=gam))
            Eg, Sx = Eg - float(src_o.flatten()[0]), Sx + float(src_o.flatten()[1])
            state["o"] = [Eg, Sx, *_gas_from_conserved(D, Eg, Sx, gam)]
            Eg, Sx, rho, p, u1 = state["g"]
            gg = {"rho": torch.full(sh, rho, dtype=torch.float64, device="cuda"),
                  "alpha_a": torch.full(sh, aa, dtype=torch.float64, device="cuda"),
                  "alpha_s": torch.zeros(sh, dtype=torch.float64, device="cuda"), "eta": None,
                  "u": torch.tensor([u1, 0.0, 0.0], dtype=torch.float64, device="cuda").expand(sh + (3,)).contiguous(),
                  "T": torch.full(sh, p / rho, dtype=torch.float64, device="cuda")}
            src_g = torch.zeros(sh + (4,), dtype=torch.float64, device="cuda")
            rad.rad_step(gc.ctx, I_g, gg, dt, rad.rad_opts_default(precision=rad.RAD_F64, gamma=gam,
                                                                   recon=rad.RAD_RECON_DC), src_g)
            sg = src_g.cpu().numpy().reshape(-1, 4)[0]
            Eg, Sx = Eg - float(sg[0]), Sx + float(sg[1])
            state["g"] = [Eg, Sx, *_gas_from_conserved(D, Eg, Sx, gam)]
        rad.rad_check(gc.ctx)
        for a, b in zip(state["g"], state["o"]):
            assert abs(a - b) <= 1e-11 * abs(b)
        assert rel_err(gc.from_gpu_I(I_g, gmap), I_o.numpy()) < 1e-11
    finally:
        gc.close()



PPM_CASES = [
    # name, sizes, level, precision, steps, C (optical depth)
    ("turb3d", (7, 5, 9), 2, "f64", 2, 0.0),            # flat 3D, periodic
    ("turb3d", (7, 5, 9), 2, "f32", 2, 0.0),
    ("turb3d", (4, 3, 37), 2, "f64", 1, 0.0),           # two x3 chunks
    ("torus3d", (8, 6, 4), 2, "f64", 2, 0.0),           # Kerr-Schild: polar (3 ghosts), outflow, angular fluxes
    ("torus3d_big", (6, 4, 4), 2, "f32", 1, 0.0),
    ("adjoint2d", (10, 8, 1), 2, "f64", 1, 0.0),        # 2D
    ("turb3d", (7, 5, 6), 2, "f64", 1, 3.0),            # with the optical-depth weighting
]


@pytest.mark.parametrize("name,n,level,prec,steps,C", PPM_CASES)
def test_ppm_step_matches_oracle(name, n, level, prec, steps, C):
    """PPM reconstruction (Colella & Woodward 1984; Sec. 2.3) against the
    oracle: FP64 1e-12, FP32 2e-5."""
    w = W.make(name, n=n, level=level)
    r = run_both(w, steps, prec, recon="ppm", tau=C)
    try:
        tol = TOL64 if prec == "f64" else TOL32
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
    finally:
        r["gc"].close()


RADDOM_CASES = [
    # name, sizes, level, precision, recon, steps
    ("turb3d", (7, 5, 6), 2, "f64", "plm", 2),          # flat, moving gas, rho spread over 1e-3 .. 10
    ("turb3d", (7, 5, 6), 2, "f32", "plm", 2),
    ("turb3d", (4, 3, 37), 2, "f64", "dc", 1),          # several chunks of cells along x3
    ("torus3d", (8, 6, 4), 2, "f64", "plm", 2),         # Kerr-Schild, gas at rest, torus density x 10
    ("torus3d_big", (6, 6, 4), 2, "f64", "dc", 1),      # moving gas and scattering in Kerr-Schild
    ("torus3d_big", (6, 6, 4), 2, "f32", "plm", 1),
]


@pytest.mark.parametrize("name,n,level,prec,recon,steps", RADDOM_CASES)
def test_radiation_dominated_substitution_matches_oracle(name, n, level, prec, recon, steps):
    """The radiation-dominated velocity substitution (end of Sec. 2.5) against
    the oracle: I and T to FP64 1e-12 / FP32 2e-5, the gas source to 1e-11
    (FP64).  The density is spread so that the substitution is active in
    some cells and not in others."""
    from oracle import coupling as OC
    from tests.harness import oracle_gas, oracle_setup
    w = W.make(name, n=n, level=level)
    if name == "turb3d":
        w["rho"] = 10.0 ** np.random.default_rng(4).uniform(-3, 1, w["T"].shape)
    else:
        w["rho"] = 10.0 * w["rho"]       # a gas-dominated core inside a radiation-dominated envelope
    st = oracle_setup(w)
    act = OC.substituted_velocity(torch.tensor(w["I0"]), torch.tensor(w["T"]), oracle_gas(w), 0.01, st)[2]
    assert 0 < int(act.sum()) < act.numel()
    r = run_both(w, steps, prec, recon=recon, rad_dom=True)
    try:
        tol = TOL64 if prec == "f64" else TOL32
        assert rel_err(r["I_g"], r["I_o"]) < tol
        assert rel_err(r["T_g"], r["T_o"]) < tol
        if prec == "f64":
            assert rel_err(r["src_g"], r["src_o"]) < 1e-11
    finally:
        r["gc"].close()
