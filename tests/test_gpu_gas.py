"""rad_gas_update (end of Sec. 2.5: the gas takes the step's -dR^0_mu)
against the oracle's gas update: random sources on a Kerr-Schild grid with
moving gas, and the moving equilibration of Sec. 3 run on the GPU (rad_step
then rad_gas_update every step) against the same loop in the oracle."""
import math
import os

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import gas as GU
from oracle import step as OS
from tests.harness import GpuCase, match_bins, oracle_setup

pytestmark = pytest.mark.gpu

F64 = torch.float64


@pytest.mark.parametrize("name", ["torus3d_big", "turb3d"])
def test_gas_update_matches_oracle(name):
    w = W.make(name, n=(6, 5, 4), level=1, with_intensity=False)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        rng = np.random.default_rng(4)
        rho, u, T = torch.tensor(w["rho"]), torch.tensor(w["u"]), torch.tensor(w["T"])
        D, Q = GU.conserved(rho, u, T, st, 5.0 / 3.0)
        src = torch.tensor(rng.normal(0.0, 0.02, (2,) + T.shape + (4,))) * Q[..., :1].abs()
        ro, uo, To, ok = GU.gas_update(rho, u, T, src.sum(0), st, 5.0 / 3.0)
        assert bool(ok.all())
        t = lambda a: a.to("cuda").contiguous()
        rg, ug, Tg = t(rho), t(u), t(T)
        rad.rad_gas_update(gc.ctx, rg, ug, Tg, t(src), 5.0 / 3.0)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert float((rg.cpu() - ro).abs().max()) <= 1e-12 * float(ro.abs().max())
        assert float((ug.cpu() - uo).abs().max()) <= 1e-12 * max(1.0, float(uo.abs().max()))
        assert float((Tg.cpu() - To).abs().max()) <= 1e-12 * float(To.abs().max())
        # a zero source leaves the state as it was
        r2, u2, T2 = t(rho), t(u), t(T)
        rad.rad_gas_update(gc.ctx, r2, u2, T2, torch.zeros_like(t(src[0])), 5.0 / 3.0)
        torch.cuda.synchronize()
        assert float((T2.cpu() - T).abs().max()) <= 1e-13 * float(T.abs().max())
    finally:
        gc.close()


def test_moving_equilibration_on_the_gpu_matches_the_oracle_loop():
    g = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "static_equilibration.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            g[k.strip()] = float(v.split()[0])
    gam, aa, p0, E0 = g["gamma"], g["alpha_a"], g["p_gas0"], g["u_rad0"]
    w = W.make("turb3d", n=(1, 1, 1), level=4, with_intensity=False)
    w["rho"] = np.full((1, 1, 1), g["rho"])
    w["u"] = np.zeros((1, 1, 1, 3))
    w["u"][..., 0] = 1.0
    w["T"] = np.full((1, 1, 1), p0 / g["rho"])
    w["alpha_a"] = np.full((1, 1, 1), aa)
    w["alpha_s"] = np.zeros((1, 1, 1))
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        na = gc.n_ang
        dt = 20.0 / 25
        I0 = np.full((1, 1, 1, na), E0 / (4 * math.pi))
        # oracle loop
        I, rho, u, T = torch.tensor(I0), torch.tensor(w["rho"]), torch.tensor(w["u"]), torch.tensor(w["T"])
        for _ in range(25):
            gas = {"rho": rho, "u": u, "alpha_a": torch.tensor(w["alpha_a"]), "alpha_s": torch.tensor(w["alpha_s"]),
                   "eta": None}
            I, _, src, ok = OS.rk2_step(I, T, gas, dt, st, OS.Opts(recon="dc", gamma=gam))
            rho, u, T, ok2 = GU.gas_update(rho, u, T, src, st, gam)
            assert bool(ok.all()) and bool(ok2.all())
        # GPU loop: rad_step, then rad_gas_update from the state the step started from
        Ig = gc.to_gpu_I(I0, gmap, F64)
        gg = gc.gas(w)
        srcg = torch.zeros((1, 1, 1, 4), dtype=F64, device="cuda")
        o = rad.rad_opts_default(recon=rad.RAD_RECON_DC, gamma=gam)
        for _ in range(25):
            T_start = gg["T"].clone()
            rad.rad_step(gc.ctx, Ig, gg, dt, o, srcg)
            gg["T"].copy_(T_start)
            rad.rad_gas_update(gc.ctx, gg["rho"], gg["u"], gg["T"], srcg, gam)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert abs(float(gg["rho"].cpu().flatten()[0]) - float(rho.flatten()[0])) < 1e-11 * float(rho.flatten()[0])
        assert float((gg["u"].cpu() - u).abs().max()) < 1e-11
        assert abs(float(gg["T"].cpu().flatten()[0]) - float(T.flatten()[0])) < 1e-11 * float(T.flatten()[0])
        assert np.abs(gc.from_gpu_I(Ig, gmap) - I.numpy()).max() < 1e-11 * np.abs(I.numpy()).max()
    finally:
        gc.close()
