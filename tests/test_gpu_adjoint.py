"""Hand-written adjoint (rad_step_adjoint) against the oracle's exact
reverse-mode gradient, and the outgoing-flux loss gradient through several
steps against central finite differences of the CUDA forward.

Tolerances: one-step vector-Jacobian products 1e-11 relative (normwise per
output, FP64); the multi-step gradient 1e-10 relative; finite differences
1e-6 relative (floored at 1e-2 of the largest gradient entry, below which the
difference quotient is roundoff-limited)."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import adjoint as OA
from oracle import cfl as OCFL
from oracle import step as OS
from paper_2302_04283_gb300.autograd import OuterLossFn, RadStepFn, StepConfig
from tests.harness import GpuCase, match_bins, oracle_gas, oracle_setup, rel_err

pytestmark = pytest.mark.gpu


def _emissivity_workload(name, n, level):
    w = W.make(name, n=n, level=level)
    if w["eta"] is None:    # give flat-space workloads an emissivity field
        rng = np.random.default_rng(17)
        w["eta"] = 10.0 ** rng.uniform(-1, 1, w["T"].shape) / (4 * np.pi)
    w["mode"] = "emissivity"
    return w


@pytest.mark.parametrize("name,n,level,recon", [
    ("adjoint2d", (10, 8, 1), 2, "plm"),
    ("adjoint2d", (7, 6, 1), 1, "dc"),
    ("torus3d", (6, 6, 4), 2, "plm"),          # Kerr-Schild 3D: polar with the pi shift in phi
    ("turb3d", (6, 5, 7), 2, "plm"),           # flat, periodic, moving gas
    ("torus3d_big", (5, 4, 4), 1, "plm"),      # moving gas and scattering in Kerr-Schild
])
def test_step_vjp_matches_oracle(name, n, level, recon):
    w = _emissivity_workload(name, n, level)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        opts = OS.Opts(recon=recon, mode="emissivity")
        rng = np.random.default_rng(5)
        lam = rng.normal(size=w["I0"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, _, ga_o, gs_o, ge_o = OA.step_vjp(I0, T0, oracle_gas(w), dt, st, opts, torch.tensor(lam))
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY,
                                 recon=rad.RAD_RECON_PLM if recon == "plm" else rad.RAD_RECON_DC)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float64)
        lg = gc.to_gpu_I(lam, gmap, torch.float64)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
        ge = torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, None, None, ga, gs, ge)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < 1e-11
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 1e-11
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 1e-11
        assert rel_err(ge.cpu().numpy(), ge_o.numpy()) < 1e-11
    finally:
        gc.close()


def _gpu_loss_and_grad(gc, w, gmap, dt, nsteps, o, fields=None):
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    aa = t(w["alpha_a"] if fields is None else fields["alpha_a"]).requires_grad_(True)
    as_ = t(w["alpha_s"] if fields is None else fields["alpha_s"]).requires_grad_(True)
    eta = t(w["eta"] if fields is None else fields["eta"]).requires_grad_(True)
    gas = gc.gas(w)
    cfg = StepConfig(gc.ctx, gas, dt, o)
    I = gc.to_gpu_I(w["I0"], gmap, torch.float64)
    for _ in range(nsteps):
        I = RadStepFn.apply(I, aa, as_, eta, cfg)
    L = OuterLossFn.apply(I, gc.ctx, rad.RAD_F64)
    L.backward()
    return float(L), aa.grad, as_.grad, eta.grad


def test_multistep_gradient_matches_oracle():
    w = _emissivity_workload("adjoint2d", (12, 8, 1), 2)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        nsteps = 4
        Lo, (ga_o, gs_o, ge_o) = OA.gradient(torch.tensor(w["I0"]), torch.tensor(w["T"]), oracle_gas(w), dt, st,
                                             OS.Opts(mode="emissivity"), nsteps)
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        L, ga, gs, ge = _gpu_loss_and_grad(gc, w, gmap, dt, nsteps, o)
        assert abs(L - float(Lo)) < 1e-12 * abs(float(Lo))
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 1e-10
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 1e-10
        assert rel_err(ge.cpu().numpy(), ge_o.numpy()) < 1e-10
    finally:
        gc.close()


def test_adjoint_workload_gradient_matches_finite_differences():
    """The 2D Kerr-Schild adjoint workload at full size (256 x 128, level 4,
    8 steps): gradient by the adjoint vs central differences of the CUDA
    forward on 16 cells drawn with the workload seed, for all three fields."""
    w = W.make("adjoint2d")
    gc = GpuCase(w)
    try:
        ang_dir = gc.dir
        gmap = np.arange(gc.n_ang)                 # inputs are generated in the library's bin order
        dt = rad.rad_cfl_dt(gc.ctx, w["cfl"])
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        L, ga, gs, ge = _gpu_loss_and_grad(gc, w, gmap, dt, w["nsteps"], o)
        grads = {"alpha_a": ga.cpu().numpy(), "alpha_s": gs.cpu().numpy(), "eta": ge.cpu().numpy()}
        cells = W.fd_cells(w, 16)

        def loss_with(field, cell, h):
            f = {k: w[k].copy() for k in ("alpha_a", "alpha_s", "eta")}
            f[field][cell] += h
            gas = gc.gas(w)
            gas.update({k: torch.tensor(v, device="cuda") for k, v in f.items()})
            I = gc.to_gpu_I(w["I0"], gmap, torch.float64)
            for _ in range(w["nsteps"]):
                rad.rad_step(gc.ctx, I, gas, dt, o)
            Ld = torch.zeros(1, dtype=torch.float64, device="cuda")
            rad.rad_loss_outer(gc.ctx, I, rad.RAD_F64, Ld)
            return float(Ld)

        for field in ("alpha_a", "alpha_s", "eta"):
            gmax = np.abs(grads[field]).max()
            for cell in cells:
                h = 1e-5 * w[field][cell]
                fd = (loss_with(field, cell, h) - loss_with(field, cell, -h)) / (2 * h)
                ad = grads[field][cell]
                assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-2 * gmax), (field, cell, fd, ad)
        assert ang_dir.shape[0] == gc.n_ang
    finally:
        gc.close()


@pytest.mark.parametrize("name,n,level", [("adjoint2d", (10, 8, 1), 2), ("torus3d", (6, 6, 4), 2)])
def test_step_vjp_f32_matches_oracle(name, n, level):
    """The FP32 adjoint against the oracle's FP64 reverse mode.  Tolerance
    2e-4 relative (normwise per output): single-precision transport and
    coupling in both the recomputed forward and the reverse sweep, and
    per-cell gradient sums over every bin."""
    w = _emissivity_workload(name, n, level)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        rng = np.random.default_rng(6)
        lam = rng.normal(size=w["I0"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, _, ga_o, gs_o, ge_o = OA.step_vjp(I0, T0, oracle_gas(w), dt, st, OS.Opts(mode="emissivity"),
                                                 torch.tensor(lam))
        o = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_EMISSIVITY)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float32)
        lg = gc.to_gpu_I(lam, gmap, torch.float32)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
        ge = torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, None, None, ga, gs, ge)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < 2e-4
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 2e-4
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 2e-4
        assert rel_err(ge.cpu().numpy(), ge_o.numpy()) < 2e-4
    finally:
        gc.close()


def _thermal_workload(name, n, level):
    w = W.make(name, n=n, level=level)
    w["mode"], w["eta"] = "thermal", None
    return w


@pytest.mark.parametrize("name,n,level,recon", [
    ("adjoint2d", (10, 8, 1), 2, "plm"),
    ("turb3d", (6, 5, 7), 2, "plm"),            # flat, periodic, moving gas
    ("torus3d", (6, 6, 4), 2, "dc"),            # Kerr-Schild 3D, polar
    ("torus3d_big", (5, 4, 4), 1, "plm"),       # moving gas and scattering in Kerr-Schild
])
def test_thermal_step_vjp_matches_oracle(name, n, level, recon):
    """Thermal coupling: the adjoint through the quartic's root and the
    temperature (lamT in and out) against the oracle's reverse mode, FP64:
    1e-11 relative per output, and 2e-10 for dL/dalpha_s, whose terms
    (through S, B0, B1 and alpha_E) cancel: on the torus case (alpha_s = 0)
    the oracle's own dL/dalpha_s moves by 2.9e-11 relative when its inputs
    are perturbed by 1e-15."""
    w = _thermal_workload(name, n, level)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        rng = np.random.default_rng(11)
        lam, lamT = rng.normal(size=w["I0"].shape), rng.normal(size=w["T"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, lamT_o, ga_o, gs_o, _ = OA.step_vjp(I0, T0, oracle_gas(w), dt, st, OS.Opts(recon=recon),
                                                   torch.tensor(lam), torch.tensor(lamT))
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_THERMAL,
                                 recon=rad.RAD_RECON_PLM if recon == "plm" else rad.RAD_RECON_DC)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float64)
        lg = gc.to_gpu_I(lam, gmap, torch.float64)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        lTg = torch.tensor(lamT, device="cuda")
        lTn = torch.zeros_like(lTg)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, lTg, lTn, ga, gs, None)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < 1e-11
        assert rel_err(lTn.cpu().numpy(), lamT_o.numpy()) < 1e-11
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 1e-11
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 2e-10
        # lamT_n may alias lamT_np1 (in place)
        ln2 = torch.zeros_like(Ig)
        ga2, gs2 = torch.zeros_like(ga), torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln2, lTg, lTg, ga2, gs2, None)
        torch.cuda.synchronize()
        assert torch.equal(lTg, lTn) and torch.equal(ln2, ln) and torch.equal(ga2, ga)
    finally:
        gc.close()


@pytest.mark.parametrize("name,n,level", [("adjoint2d", (10, 8, 1), 2), ("torus3d", (6, 6, 4), 2)])
def test_thermal_step_vjp_f32_matches_oracle(name, n, level):
    """The FP32 thermal adjoint against the oracle's FP64 reverse mode;
    tolerance 2e-4 relative per output, as for the fixed-emissivity FP32
    adjoint (the per-cell chain through the quartic is FP64 on both sides)."""
    w = _thermal_workload(name, n, level)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        rng = np.random.default_rng(12)
        lam, lamT = rng.normal(size=w["I0"].shape), rng.normal(size=w["T"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, lamT_o, ga_o, gs_o, _ = OA.step_vjp(I0, T0, oracle_gas(w), dt, st, OS.Opts(),
                                                   torch.tensor(lam), torch.tensor(lamT))
        o = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_THERMAL)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float32)
        lg = gc.to_gpu_I(lam, gmap, torch.float32)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        lTg = torch.tensor(lamT, device="cuda")
        lTn = torch.zeros_like(lTg)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, lTg, lTn, ga, gs, None)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < 2e-4
        assert rel_err(lTn.cpu().numpy(), lamT_o.numpy()) < 2e-4
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < 2e-4
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < 2e-4
    finally:
        gc.close()


def test_thermal_multistep_gradient_matches_oracle():
    """dL/d(alpha_a, alpha_s, T^0) of the outgoing-flux loss after 4 thermal
    steps, through torch.autograd (RadStepThermalFn) on the GPU, against the
    oracle's chained reverse mode; 1e-10 relative."""
    from paper_2302_04283_gb300.autograd import RadStepThermalFn
    from tests.test_oracle_moments_cfl_adjoint import _chain_vjp
    w = _thermal_workload("adjoint2d", (12, 8, 1), 2)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        nsteps = 4
        Lo, _, lamT_o, ga_o, gs_o = _chain_vjp(torch.tensor(w["I0"]), torch.tensor(w["T"]), oracle_gas(w), dt, st,
                                               OS.Opts(), nsteps)
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_THERMAL)
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        aa, as_, T = t(w["alpha_a"]).requires_grad_(True), t(w["alpha_s"]).requires_grad_(True), \
            t(w["T"]).requires_grad_(True)
        cfg = StepConfig(gc.ctx, gc.gas(w), dt, o)
        I, Tc = gc.to_gpu_I(w["I0"], gmap, torch.float64), T
        for _ in range(nsteps):
            I, Tc = RadStepThermalFn.apply(I, Tc, aa, as_, cfg)
        L = OuterLossFn.apply(I, gc.ctx, rad.RAD_F64)
        L.backward()
        rad.rad_check(gc.ctx)
        assert abs(float(L) - Lo) < 1e-12 * abs(Lo)
        assert rel_err(aa.grad.cpu().numpy(), ga_o.numpy()) < 1e-10
        assert rel_err(as_.grad.cpu().numpy(), gs_o.numpy()) < 1e-10
        assert rel_err(T.grad.cpu().numpy(), lamT_o.numpy()) < 1e-10
    finally:
        gc.close()


def test_frozen_temperature_passes_its_adjoint_through():
    """Fixed-emissivity coupling leaves T unchanged, so lamT_n = lamT_np1
    (and a NULL lamT_np1 gives zero)."""
    w = _emissivity_workload("adjoint2d", (7, 6, 1), 1)
    gc = GpuCase(w)
    try:
        dt = rad.rad_cfl_dt(gc.ctx, w["cfl"])
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        gmap = np.arange(gc.n_ang)
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float64)
        lg = torch.ones_like(Ig)
        gas = gc.gas(w)
        lTg = torch.tensor(np.random.default_rng(3).normal(size=w["T"].shape), device="cuda")
        lTn = torch.full_like(lTg, 7.0)
        z = torch.zeros_like(gas["rho"])
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, torch.zeros_like(Ig), lTg, lTn, z, z.clone(), None)
        torch.cuda.synchronize()
        assert torch.equal(lTn, lTg)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, torch.zeros_like(Ig), None, lTn, z, z.clone(), None)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        assert float(lTn.abs().max()) == 0.0
    finally:
        gc.close()


def _moving(w, seed=8, vmax=0.3):
    """Give a gas at rest random velocities (the optical-depth weighting acts
    only across velocity differences)."""
    if not np.any(w["u"]):
        rng = np.random.default_rng(seed)
        v = rng.uniform(-1, 1, w["u"].shape)
        v *= vmax / np.sqrt((v * v).sum(-1)).max()
        w["u"] = v / np.sqrt(1 - (v * v).sum(-1))[..., None]
    return w


TAU_ADJ_CASES = [
    # name, sizes, level, recon, coupling, C, precision
    ("turb3d", (6, 5, 7), 2, "plm", "emissivity", 3.0, "f64"),      # flat, periodic
    ("turb3d", (5, 4, 6), 2, "dc", "emissivity", 10.0, "f64"),
    ("adjoint2d", (9, 8, 1), 2, "plm", "emissivity", 5.0, "f64"),   # 2D Kerr-Schild, outflow
    ("torus3d_big", (5, 4, 4), 1, "plm", "emissivity", 20.0, "f64"),  # polar with the pi shift, scattering
    ("torus3d_big", (5, 4, 4), 1, "plm", "thermal", 20.0, "f64"),
    ("turb3d", (6, 5, 7), 2, "plm", "emissivity", 3.0, "f32"),
]


@pytest.mark.parametrize("name,n,level,recon,coupling,C,prec", TAU_ADJ_CASES)
def test_tau_weighted_step_vjp_matches_oracle(name, n, level, recon, coupling, C, prec):
    """The adjoint with the optical-depth weighting of Sec. 2.4 against the
    oracle's reverse mode: every output at 1e-11 (FP64; 2e-10 for the thermal
    dL/dalpha_s as without the weighting) or 2e-4 (FP32), and the weighting's
    own share of the opacity gradients (the difference from the unweighted
    adjoint, run on both sides) at 1e-8 of its norm in FP64."""
    w = _thermal_workload(name, n, level) if coupling == "thermal" else _emissivity_workload(name, n, level)
    w = _moving(w)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        rng = np.random.default_rng(12)
        lam = rng.normal(size=w["I0"].shape)
        lamT = rng.normal(size=w["T"].shape) if coupling == "thermal" else None
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        f64 = prec == "f64"
        tdt = torch.float64 if f64 else torch.float32
        out = {}
        for CC in (C, 0.0):
            lam_o, lamT_o, ga_o, gs_o, _ = OA.step_vjp(I0, T0, oracle_gas(w), dt, st,
                                                       OS.Opts(recon=recon, mode=coupling, tau_const=CC),
                                                       torch.tensor(lam),
                                                       None if lamT is None else torch.tensor(lamT))
            o = rad.rad_opts_default(precision=rad.RAD_F64 if f64 else rad.RAD_F32,
                                     coupling=rad.RAD_COUPLE_THERMAL if coupling == "thermal"
                                     else rad.RAD_COUPLE_EMISSIVITY,
                                     recon=rad.RAD_RECON_PLM if recon == "plm" else rad.RAD_RECON_DC, tau_const=CC)
            Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
            lg = gc.to_gpu_I(lam, gmap, tdt)
            ln = torch.zeros_like(Ig)
            gas = gc.gas(w)
            lTg = None if lamT is None else torch.tensor(lamT, device="cuda")
            lTn = None if lamT is None else torch.zeros_like(lTg)
            ga = torch.zeros_like(gas["rho"])
            gs = torch.zeros_like(ga)
            ge = torch.zeros_like(ga) if coupling == "emissivity" else None
            rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, lTg, lTn, ga, gs, ge)
            torch.cuda.synchronize()
            rad.rad_check(gc.ctx)
            out[CC] = (gc.from_gpu_I(ln.double(), gmap), ga.cpu().numpy(), gs.cpu().numpy(),
                       lam_o.numpy(), ga_o.numpy(), gs_o.numpy(),
                       None if lTn is None else (lTn.cpu().numpy(), lamT_o.numpy()))
        lg_, ga_, gs_, lo_, gao, gso, lt = out[C]
        tol = 1e-11 if f64 else 2e-4
        assert rel_err(lg_, lo_) < tol
        assert rel_err(ga_, gao) < tol
        assert rel_err(gs_, gso) < (2e-10 if f64 and coupling == "thermal" else tol)
        if lt is not None:
            assert rel_err(lt[0], lt[1]) < tol
        # the weighting's own share of the opacity gradients (FP64: in FP32 the
        # share is below the rounding of the totals)
        _, ga0, gs0, _, gao0, gso0, _ = out[0.0]
        dgo = gao - gao0
        assert np.abs(dgo).max() > 1e-4 * np.abs(gao).max()     # the weighting matters here
        if f64:
            assert rel_err(ga_ - ga0, dgo) < 1e-8
            # thermal dL/dalpha_s: its conditioning (2.9e-11 of the total, see
            # above) over the weighting's share (~2e-4 of it)
            assert rel_err(gs_ - gs0, gso - gso0) < (1e-6 if coupling == "thermal" else 1e-8)
    finally:
        gc.close()


PPM_ADJ_CASES = [
    # name, sizes, level, recon, coupling, C, precision
    ("turb3d", (7, 6, 7), 2, "ppm", "emissivity", 0.0, "f64"),       # flat, periodic
    ("adjoint2d", (10, 8, 1), 2, "ppm", "emissivity", 0.0, "f64"),   # 2D Kerr-Schild, outflow
    ("torus3d", (6, 6, 4), 2, "ppm", "emissivity", 0.0, "f64"),      # polar, and a 4-cell periodic x3
    ("torus3d", (5, 3, 4), 1, "ppm", "emissivity", 0.0, "f64"),      # three rows: stencils cross both poles
    ("torus3d_big", (5, 4, 4), 1, "ppm", "thermal", 0.0, "f64"),     # moving gas, scattering
    ("turb3d", (5, 4, 6), 2, "ppm", "emissivity", 0.0, "f64"),       # periodic lines shorter than the window
    ("turb3d", (3, 4, 5), 2, "plm", "emissivity", 0.0, "f64"),       # the same for PLM (3 < 4 faces)
    ("torus3d", (5, 2, 4), 1, "plm", "emissivity", 0.0, "f64"),      # two rows: the window reaches past both poles
    ("turb3d", (6, 5, 7), 2, "ppm", "emissivity", 3.0, "f64"),       # with the optical-depth weighting
    ("turb3d", (7, 6, 7), 2, "ppm", "emissivity", 0.0, "f32"),
]


@pytest.mark.parametrize("name,n,level,recon,coupling,C,prec", PPM_ADJ_CASES)
def test_ppm_step_vjp_matches_oracle(name, n, level, recon, coupling, C, prec):
    """The adjoint with PPM reconstruction (and short periodic lines, where a
    face appears twice in the gather window) against the oracle's reverse
    mode: FP64 1e-11 per output (thermal dL/dalpha_s 2e-10), FP32 2e-4."""
    w = _thermal_workload(name, n, level) if coupling == "thermal" else _emissivity_workload(name, n, level)
    if C > 0:
        w = _moving(w)
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        rng = np.random.default_rng(13)
        lam = rng.normal(size=w["I0"].shape)
        lamT = rng.normal(size=w["T"].shape) if coupling == "thermal" else None
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, lamT_o, ga_o, gs_o, ge_o = OA.step_vjp(I0, T0, oracle_gas(w), dt, st,
                                                      OS.Opts(recon=recon, mode=coupling, tau_const=C),
                                                      torch.tensor(lam), None if lamT is None else torch.tensor(lamT))
        f64 = prec == "f64"
        tdt = torch.float64 if f64 else torch.float32
        o = rad.rad_opts_default(precision=rad.RAD_F64 if f64 else rad.RAD_F32,
                                 coupling=rad.RAD_COUPLE_THERMAL if coupling == "thermal" else rad.RAD_COUPLE_EMISSIVITY,
                                 recon={"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM}[recon],
                                 tau_const=C)
        Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
        lg = gc.to_gpu_I(lam, gmap, tdt)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        lTg = None if lamT is None else torch.tensor(lamT, device="cuda")
        lTn = None if lamT is None else torch.zeros_like(lTg)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
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



@pytest.mark.parametrize("name,n,level,prec,recon", [
    ("turb3d", (7, 5, 6), 2, "f64", "plm"),          # flat, moving gas, rho spread over 1e-3 .. 10
    ("turb3d", (4, 3, 9), 2, "f64", "dc"),
    ("torus3d", (8, 6, 4), 2, "f64", "plm"),         # Kerr-Schild, gas at rest, torus density x 10
    ("torus3d_big", (6, 6, 4), 2, "f64", "plm"),     # moving gas and scattering in Kerr-Schild
    ("turb3d", (7, 5, 6), 2, "f32", "plm"),
])
def test_radiation_dominated_step_vjp_matches_oracle(name, n, level, prec, recon):
    """rad_dom = 1: the adjoint through the substituted velocity against the
    oracle's reverse mode (FP64 1e-11, dL/dalpha_s 2e-10 as for the thermal
    adjoint; FP32 2e-4).  The density is spread so that the substitution is
    active in some cells and not in others."""
    from oracle import coupling as OC
    w = _thermal_workload(name, n, level)
    if name == "turb3d":
        w["rho"] = 10.0 ** np.random.default_rng(4).uniform(-3, 1, w["T"].shape)
    else:
        w["rho"] = 10.0 * w["rho"]
    st = oracle_setup(w)
    gc = GpuCase(w)
    try:
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        dt = OCFL.cfl_dt(st, w["cfl"])
        act = OC.substituted_velocity(torch.tensor(w["I0"]), torch.tensor(w["T"]), oracle_gas(w), dt, st)[2]
        assert 0 < int(act.sum()) < act.numel()
        rng = np.random.default_rng(13)
        lam, lamT = rng.normal(size=w["I0"].shape), rng.normal(size=w["T"].shape)
        I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
        lam_o, lamT_o, ga_o, gs_o, _ = OA.step_vjp(I0, T0, oracle_gas(w), dt, st,
                                                   OS.Opts(recon=recon, rad_dom=True),
                                                   torch.tensor(lam), torch.tensor(lamT))
        f32 = prec == "f32"
        tdt = torch.float32 if f32 else torch.float64
        o = rad.rad_opts_default(precision=rad.RAD_F32 if f32 else rad.RAD_F64, coupling=rad.RAD_COUPLE_THERMAL,
                                 recon=rad.RAD_RECON_PLM if recon == "plm" else rad.RAD_RECON_DC, rad_dom=1)
        Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
        lg = gc.to_gpu_I(lam, gmap, tdt)
        ln = torch.zeros_like(Ig)
        gas = gc.gas(w)
        lTg = torch.tensor(lamT, device="cuda")
        lTn = torch.zeros_like(lTg)
        ga = torch.zeros_like(gas["rho"])
        gs = torch.zeros_like(ga)
        rad.rad_step_adjoint(gc.ctx, Ig, gas, dt, o, lg, ln, lTg, lTn, ga, gs, None)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        tol = 2e-4 if f32 else 1e-11
        assert rel_err(gc.from_gpu_I(ln, gmap), lam_o.numpy()) < tol
        assert rel_err(lTn.cpu().numpy(), lamT_o.numpy()) < tol
        assert rel_err(ga.cpu().numpy(), ga_o.numpy()) < tol
        assert rel_err(gs.cpu().numpy(), gs_o.numpy()) < (2e-4 if f32 else 2e-10)
    finally:
        gc.close()
