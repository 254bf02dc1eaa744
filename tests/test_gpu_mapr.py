"""Minimum-angle plane reconstruction (MAPR) of the angular face values on
geodesic grids (recon_ang = RAD_RECON_MAPR) through the C ABI, against the
oracle: FP64 1e-12, FP32 2e-5 relative (normwise per output), as for every
step; and the options that refuse it."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from tests.harness import GpuCase, rel_err, run_both

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
        with pytest.raises(rad.RadError) as e:           # the adjoint does not cover it
            rad.rad_step_adjoint(gc.ctx, I, gc.gas(w), 0.01,
                                 rad.rad_opts_default(coupling=rad.RAD_COUPLE_NONE, recon_ang=rad.RAD_RECON_MAPR),
                                 I, torch.zeros_like(I), None, None, z, z.clone())
        assert e.value.status == rad.RAD_EUNSUPPORTED
        with pytest.raises(rad.RadError) as e:           # as a spatial reconstruction it is unknown
            rad.rad_step(gc.ctx, I, gc.gas(w), 0.01, rad.rad_opts_default(recon=rad.RAD_RECON_MAPR))
        assert e.value.status == rad.RAD_EINVAL
    finally:
        gc.close()
