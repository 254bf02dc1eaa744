"""Multigroup transport through the C ABI (rad_set_groups, rad_step) against
the oracle's (Sec. 2.2, Eq. radiation_integral_frequency): the frequency
fluxes of the redshift term, donor cell in frequency, with per-group
fixed-emissivity coupling, on Kerr-Schild grids where omega^0hat does not
vanish.  Tolerances as the gray parity tests: FP64 1e-12, FP32 2e-5
(normwise per output)."""
import math

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import cfl as OCFL
from oracle import frequency as FQ
from oracle import step as OS
from tests.harness import GpuCase, match_bins, oracle_setup, rel_err

pytestmark = pytest.mark.gpu

INF = float("inf")
R = {"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM, "mapr": rad.RAD_RECON_MAPR}


def _inputs(w, G_, seed):
    rng = np.random.default_rng(seed)
    sh = w["T"].shape
    aa = w["alpha_a"][None] * rng.uniform(0.5, 2.0, (G_,) + sh)
    as_ = (w["alpha_s"] + 0.1)[None] * rng.uniform(0.5, 2.0, (G_,) + sh)
    eta = rng.uniform(0.005, 0.05, (G_,) + sh)
    I0 = w["I0"][None] * rng.uniform(0.5, 1.5, (G_,) + w["I0"].shape)
    return aa, as_, eta, I0


def _run(name, n, level, edges, prec, recon, recon_ang, couple, steps, seed=7):
    w = W.make(name, n=n, level=level)
    G_ = len(edges) - 1
    aa, as_, eta, I0 = _inputs(w, G_, seed)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        rad.rad_set_groups(gc.ctx, edges)
        dt = 0.5 * rad.rad_cfl_dt(gc.ctx, w["cfl"])
        # oracle
        o = OS.Opts(recon=recon, recon_ang=recon_ang, mode="emissivity", couple=couple)
        gas_o = {"rho": torch.tensor(w["rho"]), "u": torch.tensor(w["u"]), "alpha_a": torch.tensor(aa),
                 "alpha_s": torch.tensor(as_), "eta": torch.tensor(eta)}
        I, T = torch.tensor(I0), torch.tensor(w["T"])
        for _ in range(steps):
            I, T, src, ok = FQ.rk2_step_groups(I, T, gas_o, dt, st, o, edges)
            assert bool(ok.all())
        # GPU
        tdt = torch.float64 if prec == "f64" else torch.float32
        Ig = gc.to_gpu_I(I0, gmap, tdt)
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        gas = {"rho": t(w["rho"]), "u": t(w["u"]), "alpha_a": t(aa), "alpha_s": t(as_), "eta": t(eta),
               "T": t(w["T"])}
        srcg = torch.zeros((G_,) + w["T"].shape + (4,), dtype=torch.float64, device="cuda")
        opts = rad.rad_opts_default(precision=rad.RAD_F64 if prec == "f64" else rad.RAD_F32, recon=R[recon],
                                    recon_ang=R[recon_ang],
                                    coupling=rad.RAD_COUPLE_EMISSIVITY if couple else rad.RAD_COUPLE_NONE)
        for _ in range(steps):
            rad.rad_step(gc.ctx, Ig, gas, dt, opts, srcg)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        return dict(I_o=I.numpy(), I_g=gc.from_gpu_I(Ig, gmap), src_o=src.numpy(), src_g=srcg.cpu().numpy(),
                    T_o=T.numpy(), T_g=gas["T"].cpu().numpy(), pad=Ig[..., gc.n_ang:], I0=I0, st=st, gc=gc)
    finally:
        gc.close()


CASES = [
    ("torus3d_big", (6, 5, 4), 2, [0.1, 0.5, 1.0, 2.0, 4.0], "f64", "plm", "dc", True, 2),
    ("torus3d_big", (6, 5, 4), 2, [0.1, 0.5, 1.0, 2.0, 4.0], "f32", "plm", "dc", True, 2),
    ("torus3d", (7, 6, 4), 2, [0.0, 1.0, 3.0, INF], "f64", "dc", "dc", False, 2),
    ("torus3d_big", (6, 5, 4), 2, [0.2, 0.4, 0.8, 1.6], "f64", "ppm", "mapr", True, 1),
    ("adjoint2d", (10, 8, 1), 2, [0.3, 1.0, 3.0], "f64", "plm", "dc", True, 2),
]


@pytest.mark.parametrize("name,n,level,edges,prec,recon,recon_ang,couple,steps", CASES)
def test_multigroup_step_matches_oracle(name, n, level, edges, prec, recon, recon_ang, couple, steps):
    r = _run(name, n, level, edges, prec, recon, recon_ang, couple, steps)
    tol = 1e-12 if prec == "f64" else 2e-5
    # the frequency fluxes moved energy between groups
    assert float(np.abs(r["I_o"] - 0).max()) > 0
    e = rel_err(r["I_g"], r["I_o"])
    assert e < tol, e
    assert rel_err(r["T_g"], r["T_o"]) < tol
    if couple:
        assert np.abs(r["src_g"] - r["src_o"]).max() <= (1e-11 if prec == "f64" else 1e-4) * \
            max(np.abs(r["src_o"]).max(), 1e-300) + (1e-13 if prec == "f64" else 1e-6) * np.abs(r["I_o"]).max()
    assert float(r["pad"].abs().max()) == 0.0 if r["pad"].numel() else True


def test_one_group_over_all_frequencies_is_the_gray_step():
    w = W.make("torus3d_big", n=(6, 5, 4), level=2)
    gc = GpuCase(w)
    try:
        dt = rad.rad_cfl_dt(gc.ctx, w["cfl"])
        o = rad.rad_opts_default(coupling=rad.RAD_COUPLE_EMISSIVITY)
        w["eta"] = np.full(w["T"].shape, 0.02)
        Ia = torch.nn.functional.pad(torch.tensor(w["I0"], device="cuda"), (0, gc.n_ap - gc.n_ang)).contiguous()
        Ib = Ia.clone()
        ga, gb = gc.gas(w), gc.gas(w)
        rad.rad_step(gc.ctx, Ia, ga, dt, o)
        rad.rad_set_groups(gc.ctx, [0.0, INF])
        assert rad.rad_cfl_dt(gc.ctx, w["cfl"]) == dt          # no finite group: no frequency bound
        rad.rad_step(gc.ctx, Ib, gb, dt, o)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert torch.equal(Ia, Ib)
    finally:
        gc.close()


def test_time_step_bound_with_groups():
    """rad_cfl_dt with groups: 0.3 min(spatial, angular, frequency) with the
    oracle's frequency bound n^0 dnu / (nu_hi |omega^0hat_{AB} n^A n^B|)."""
    w = W.make("torus3d_big", n=(6, 5, 4), level=2, with_intensity=False)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        edges = [1.0, 1.01, 1.02, 2.0]
        rad.rad_set_groups(gc.ctx, edges)
        got = rad.rad_cfl_dt(gc.ctx, 0.3)
        want = 0.3 * min(OCFL.cfl_dt(st, 1.0), FQ.frequency_dt(st, edges))
        assert FQ.frequency_dt(st, edges) < OCFL.cfl_dt(st, 1.0)     # the frequency bound binds here
        assert abs(got - want) <= 1e-12 * want
    finally:
        gc.close()


def test_multigroup_refusals():
    w = W.make("torus3d", n=(6, 5, 4), level=1, with_intensity=False)
    gc = GpuCase(w)
    try:
        with pytest.raises(rad.RadError):
            rad.rad_set_groups(gc.ctx, [1.0, 0.5])                   # edges must increase
        rad.rad_set_groups(gc.ctx, [0.0, 1.0, 2.0])
        I = torch.zeros((2,) + w["T"].shape + (gc.n_ap,), dtype=torch.float64, device="cuda")
        g = gc.gas(w)
        with pytest.raises(rad.RadError) as e:
            rad.rad_step(gc.ctx, I, g, 1e-3, rad.rad_opts_default())  # thermal coupling
        assert e.value.status == rad.RAD_EUNSUPPORTED
        rad.rad_set_groups(gc.ctx, [])                                # back to gray
        I1 = I[0].contiguous()
        rad.rad_step(gc.ctx, I1, g, 1e-4, rad.rad_opts_default(coupling=rad.RAD_COUPLE_NONE))
        rad.rad_check(gc.ctx)
    finally:
        gc.close()
