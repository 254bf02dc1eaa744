"""Pins of the oracle's moments (Sec. 2.5, the definition of R), its
time-step bound, and its reverse-mode gradient (checked against central
finite differences and by a dot-product test)."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import cfl as CF
from oracle import moments as M
from oracle import step as S
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup

F64 = torch.float64


def test_isotropic_moments_are_diagonal():
    for N in (1, 2, 4):
        ang = GeodesicGrid(N)
        I = torch.full((2, 3, ang.n_ang), 0.25, dtype=F64)
        R = M.moments(I, ang)
        E = 0.25 * 4 * math.pi
        ref = torch.tensor([E, 0, 0, 0, E / 3, 0, 0, E / 3, 0, E / 3], dtype=F64)
        assert (R - ref).abs().max() < 1e-14


def test_fluid_frame_energy_identity():
    """R^{0bar 0bar} = sum Ihat (n^0bar)^2 dOmega (the E-bar of Sec. 2.5)."""
    ang = GeodesicGrid(3)
    rng = np.random.default_rng(4)
    I = torch.tensor(rng.uniform(0, 1, (5, ang.n_ang)))
    u = torch.tensor(rng.uniform(-0.5, 0.5, (5, 3)))
    R = M.moments(I, ang, "fluid", u=u)
    u0 = torch.sqrt(1 + (u * u).sum(-1))
    nb = u0[:, None] - u @ ang.dir.T
    assert (R[:, 0] - (I * nb ** 2 * ang.dOmega).sum(-1)).abs().max() < 1e-14
    # the boost is a Lorentz transformation: eta-trace of R is invariant
    Rt = M.moments(I, ang)
    tr = lambda X: -X[:, 0] + X[:, 4] + X[:, 7] + X[:, 9]
    assert (tr(R) - tr(Rt)).abs().max() < 1e-13
    assert tr(Rt).abs().max() < 1e-14 * float(Rt[:, 0].max())    # null directions: traceless


def test_coordinate_frame_in_cartesian_minkowski_is_tetrad_frame():
    ang = GeodesicGrid(2)
    I = torch.rand(3, ang.n_ang, dtype=F64)
    e = torch.eye(4, dtype=F64).expand(3, 4, 4)
    assert (M.moments(I, ang, "coord", e=e) - M.moments(I, ang)).abs().max() == 0.0


def test_cfl_in_cartesian_minkowski():
    ang = GeodesicGrid(2)
    xf = [np.linspace(0, 1, 9), np.linspace(0, 2, 9), np.array([0.0, 1.0])]
    st = Setup(Grid("mink_cart", 0.0, xf, (("periodic", "periodic"),) * 3, 2), ang)
    ref = 0.3 * min(1 / 8 / float(ang.dir[:, 0].abs().max()), 2 / 8 / float(ang.dir[:, 1].abs().max()))
    assert abs(CF.cfl_dt(st, 0.3) - ref) < 1e-15


@pytest.fixture(scope="module")
def adj_case():
    w = W.make("adjoint2d", n=(6, 4, 1), level=1)
    ang = GeodesicGrid(w["level"])
    st = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), ang)
    gas = {k: (torch.tensor(w[k]) if w[k] is not None else None)
           for k in ("rho", "u", "alpha_a", "alpha_s", "eta")}
    dt = CF.cfl_dt(st, 0.3)
    return w, st, gas, dt


def test_gradient_matches_central_differences(adj_case):
    w, st, gas, dt = adj_case
    opts = S.Opts(mode="emissivity")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 3
    L, grads = A.gradient(I0, T0, gas, dt, st, opts, nsteps)

    def loss_with(field, cell, h):
        g2 = {k: (v.clone() if v is not None else None) for k, v in gas.items()}
        g2[field][cell] += h
        I, T = I0, T0
        for _ in range(nsteps):
            I, T, _, _ = S.rk2_step(I, T, g2, dt, st, opts)
        return float(A.loss_outer(I, st))

    for fi, field in enumerate(("alpha_a", "alpha_s", "eta")):
        for cell in [(0, 1, 5), (0, 2, 4), (0, 0, 3)]:
            h = 1e-5 * float(gas[field][cell])
            fd = (loss_with(field, cell, h) - loss_with(field, cell, -h)) / (2 * h)
            ad = float(grads[fi][cell])
            # relative to the gradient, floored at 2e-2 of its largest entry
            # (below that the difference quotient is limited by roundoff)
            assert abs(fd - ad) <= 1e-6 * max(abs(ad), 2e-2 * float(grads[fi].abs().max()))


def test_step_vjp_dot_product(adj_case):
    """<lambda, J delta> = <J^T lambda, delta> with J delta by forward-mode AD."""
    w, st, gas, dt = adj_case
    opts = S.Opts(mode="emissivity")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    rng = np.random.default_rng(8)
    lam = torch.tensor(rng.normal(size=I0.shape))
    dI = torch.tensor(rng.normal(size=I0.shape))
    da = torch.tensor(rng.normal(size=T0.shape))
    lam_n, _, g_aa, _, _ = A.step_vjp(I0, T0, gas, dt, st, opts, lam)

    def f(I, aa):
        g2 = dict(gas)
        g2["alpha_a"] = aa
        return S.rk2_step(I, T0, g2, dt, st, opts)[0]

    _, jvp = torch.func.jvp(f, (I0, gas["alpha_a"]), (dI, da))
    lhs = float((lam * jvp).sum())
    rhs = float((lam_n * dI).sum() + (g_aa * da).sum())
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def _chain_vjp(I0, T0, gas, dt, st, opts, nsteps):
    """dL/d(I0, T0, alpha_a, alpha_s) of the outgoing-flux loss after nsteps,
    by chaining one-step vector-Jacobian products backwards (lamT carries
    the gradient through the gas temperature)."""
    Is, Ts = [I0], [T0]
    for _ in range(nsteps):
        I, T, _, ok = S.rk2_step(Is[-1], Ts[-1], gas, dt, st, opts)
        assert ok.all()
        Is.append(I)
        Ts.append(T)
    lam, lamT = A.loss_seed(Is[-1], st), torch.zeros_like(T0)
    ga, gs = torch.zeros_like(T0), torch.zeros_like(T0)
    for s in reversed(range(nsteps)):
        lam, lamT, g1, g2, _ = A.step_vjp(Is[s], Ts[s], gas, dt, st, opts, lam, lamT)
        ga, gs = ga + g1, gs + g2
    return float(A.loss_outer(Is[-1], st)), lam, lamT, ga, gs


def test_thermal_gradient_matches_central_differences(adj_case):
    """Thermal coupling: the temperature evolves through the quartic of
    Sec. 2.5, so the gradient runs through its root (implicit-function
    theorem) and through T from step to step.  Chained one-step VJPs
    against central differences of the forward oracle for alpha_a, alpha_s
    and the initial T, and against reverse-mode AD through all steps."""
    w, st, gas, dt = adj_case
    opts = S.Opts(mode="thermal")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 3
    L, lam, lamT, ga, gs = _chain_vjp(I0, T0, gas, dt, st, opts, nsteps)
    L2, grads2 = A.gradient(I0, T0, gas, dt, st, opts, nsteps)
    ga2, gs2 = grads2[0], grads2[1]
    assert abs(L - float(L2)) <= 1e-14 * abs(L)
    assert float((ga - ga2).abs().max()) <= 1e-12 * float(ga2.abs().max())
    assert float((gs - gs2).abs().max()) <= 1e-12 * float(gs2.abs().max())

    def loss_with(field, cell, h):
        g2 = {k: (v.clone() if v is not None else None) for k, v in gas.items()}
        T = T0.clone()
        if field == "T":
            T[cell] += h
        else:
            g2[field][cell] += h
        I = I0
        for _ in range(nsteps):
            I, T, _, _ = S.rk2_step(I, T, g2, dt, st, opts)
        return float(A.loss_outer(I, st))

    for field, grad, base in (("alpha_a", ga, gas["alpha_a"]), ("alpha_s", gs, gas["alpha_s"]), ("T", lamT, T0)):
        assert float(grad.abs().max()) > 0.0
        for cell in [(0, 1, 5), (0, 2, 4), (0, 0, 3), (0, 3, 0)]:
            # relative step 1e-4: roundoff (eps |L| / h) would dominate the
            # small entries at 1e-5, and at 1e-3 a perturbation of T can
            # cross a kink of the PLM limiter
            h = 1e-4 * float(base[cell])
            fd = (loss_with(field, cell, h) - loss_with(field, cell, -h)) / (2 * h)
            ad = float(grad[cell])
            assert abs(fd - ad) <= 1e-6 * max(abs(ad), 2e-2 * float(grad.abs().max())), (field, cell, fd, ad)


def test_thermal_step_vjp_dot_product(adj_case):
    """<(lam, lamT), J (dI, dT, dalpha)> = <J^T (lam, lamT), (dI, dT, dalpha)>
    for the thermal step, with J (.) by forward-mode AD."""
    w, st, gas, dt = adj_case
    opts = S.Opts(mode="thermal")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    rng = np.random.default_rng(9)
    lam, lamT = torch.tensor(rng.normal(size=I0.shape)), torch.tensor(rng.normal(size=T0.shape))
    dI, dT = torch.tensor(rng.normal(size=I0.shape)), torch.tensor(rng.normal(size=T0.shape))
    da, ds = torch.tensor(rng.normal(size=T0.shape)), torch.tensor(rng.normal(size=T0.shape))
    lam_n, lamT_n, g_aa, g_as, _ = A.step_vjp(I0, T0, gas, dt, st, opts, lam, lamT)

    def f(I, T, aa, a_s):
        g2 = dict(gas)
        g2["alpha_a"], g2["alpha_s"] = aa, a_s
        I2, T2, _, _ = S.rk2_step(I, T, g2, dt, st, opts)
        return I2, T2

    _, (jI, jT) = torch.func.jvp(f, (I0, T0, gas["alpha_a"], gas["alpha_s"]), (dI, dT, da, ds))
    lhs = float((lam * jI).sum() + (lamT * jT).sum())
    rhs = float((lam_n * dI).sum() + (lamT_n * dT).sum() + (g_aa * da).sum() + (g_as * ds).sum())
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_tau_weighted_gradient_matches_central_differences(adj_case):
    """With the optical-depth weighting of Sec. 2.4 the face factors depend on
    alpha_E = alpha_a + alpha_s, so the opacity gradient has a second path
    (through f = -expm1(-tau^2)).  Reverse-mode AD of the oracle against
    central differences of its forward over two steps, on a moving gas (the
    weighting acts only across velocity differences); the weighting changes
    the gradient at the cells checked by far more than the tolerance, so a
    dropped path fails."""
    w, st, gas, dt = adj_case
    rng = np.random.default_rng(21)
    v = rng.uniform(-1, 1, gas["alpha_a"].shape + (3,))
    v *= 0.3 / np.sqrt((v * v).sum(-1)).max()
    g0 = dict(gas)
    g0["u"] = torch.tensor(v / np.sqrt(1 - (v * v).sum(-1))[..., None])
    opts = S.Opts(mode="emissivity", tau_const=5.0)
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 2
    L, grads = A.gradient(I0, T0, g0, dt, st, opts, nsteps)
    _, grads_free = A.gradient(I0, T0, g0, dt, st, S.Opts(mode="emissivity"), nsteps)

    def loss_with(field, cell, h):
        g2 = {k: (x.clone() if x is not None else None) for k, x in g0.items()}
        g2[field][cell] += h
        I, T = I0, T0
        for _ in range(nsteps):
            I, T, _, _ = S.rk2_step(I, T, g2, dt, st, opts)
        return float(A.loss_outer(I, st))

    for fi, field in enumerate(("alpha_a", "alpha_s")):
        gmax = float(grads[fi].abs().max())
        diff = (grads[fi] - grads_free[fi]).abs()
        # the three cells where the weighting moves the gradient most, and two more
        top = [tuple(int(x) for x in np.unravel_index(q, diff.shape)) for q in
               torch.argsort(diff.flatten(), descending=True)[:3].tolist()]
        for cell in top + [(0, 2, 4), (0, 3, 1)]:
            ad = float(grads[fi][cell])
            tol = 1e-6 * max(abs(ad), 2e-2 * gmax)
            if cell in top:
                assert float(diff[cell]) > 20 * tol, (field, cell)
            h = 1e-5 * float(g0[field][cell])
            fd = (loss_with(field, cell, h) - loss_with(field, cell, -h)) / (2 * h)
            assert abs(fd - ad) <= tol, (field, cell, fd, ad)


def test_ppm_gradient_matches_central_differences(adj_case):
    """PPM reconstruction (Colella & Woodward 1984; Sec. 2.3): its face states
    are piecewise linear in the five cells around the upwind cell, so the
    step's gradient exists away from the branch switches of its limiters.
    Reverse-mode AD of the oracle against central differences of its forward
    for alpha_a, alpha_s and the initial intensity over two steps."""
    w, st, gas, dt = adj_case
    opts = S.Opts(mode="emissivity", recon="ppm")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 2
    L, grads = A.gradient(I0, T0, gas, dt, st, opts, nsteps)
    I0r = I0.clone().requires_grad_(True)
    I = I0r
    T = T0
    for _ in range(nsteps):
        I, T, _, _ = S.rk2_step(I, T, gas, dt, st, opts)
    gI = torch.autograd.grad(A.loss_outer(I, st), I0r)[0]

    def loss_with(field, idx, h):
        g2 = {k: (x.clone() if x is not None else None) for k, x in gas.items()}
        Iv = I0.clone()
        if field == "I":
            Iv[idx] += h
        else:
            g2[field][idx] += h
        Iv2, T2 = Iv, T0
        for _ in range(nsteps):
            Iv2, T2, _, _ = S.rk2_step(Iv2, T2, g2, dt, st, opts)
        return float(A.loss_outer(Iv2, st))

    checks = [("alpha_a", grads[0], gas["alpha_a"], (0, 1, 5)), ("alpha_a", grads[0], gas["alpha_a"], (0, 2, 3)),
              ("alpha_s", grads[1], gas["alpha_s"], (0, 2, 4)), ("alpha_s", grads[1], gas["alpha_s"], (0, 3, 2))]
    # intensities two to three cells from the outer face reach it through the
    # wide PPM stencil only
    for idx in [(0, 1, 3, 4), (0, 2, 2, 7), (0, 0, 4, 1)]:
        checks.append(("I", gI, I0, idx))
    for field, grad, base, idx in checks:
        gmax = float(grad.abs().max())
        assert gmax > 0.0
        h = 1e-5 * max(abs(float(base[idx])), 1e-3 * float(base.abs().max()))
        fd = (loss_with(field, idx, h) - loss_with(field, idx, -h)) / (2 * h)
        ad = float(grad[idx])
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 2e-2 * gmax), (field, idx, fd, ad)


def test_angular_plm_gradient_matches_central_differences():
    """PLM angular reconstruction along the lines of a latitude-longitude grid
    (Sec. 2.6): each side's upwind state reads the upwind cell, the cell
    behind it on the line and the downwind cell.  Reverse-mode AD of the
    oracle against central differences of its forward on a 2D Kerr-Schild
    grid (a 3 x 6 angle grid, whose lines cross the poles), in alpha_a,
    alpha_s and in intensities of bins that enter fluxes only as cells behind."""
    from oracle.angles import LatLongGrid
    w = W.make("adjoint2d", n=(6, 4, 1), level=1, latlong=(3, 6))
    ang = LatLongGrid(3, 6)
    st = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), ang)
    gas = {k: (torch.tensor(w[k]) if w[k] is not None else None)
           for k in ("rho", "u", "alpha_a", "alpha_s", "eta")}
    dt = CF.cfl_dt(st, 0.3)
    opts = S.Opts(mode="emissivity", recon_ang="plm")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 2
    L, grads = A.gradient(I0, T0, gas, dt, st, opts, nsteps)

    def grad_I(o):
        I0r = I0.clone().requires_grad_(True)
        I, T = I0r, T0
        for _ in range(nsteps):
            I, T, _, _ = S.rk2_step(I, T, gas, dt, st, o)
        return torch.autograd.grad(A.loss_outer(I, st), I0r)[0]

    gI, gI_dc = grad_I(opts), grad_I(S.Opts(mode="emissivity"))

    def loss_with(field, idx, h):
        g2 = {k: (x.clone() if x is not None else None) for k, x in gas.items()}
        Iv = I0.clone()
        if field == "I":
            Iv[idx] += h
        else:
            g2[field][idx] += h
        Iv2, T2 = Iv, T0
        for _ in range(nsteps):
            Iv2, T2, _, _ = S.rk2_step(Iv2, T2, g2, dt, st, opts)
        return float(A.loss_outer(Iv2, st))

    # the angular reconstruction changes the gradient
    assert float((gI - gI_dc).abs().max()) > 1e-3 * float(gI.abs().max())
    checks = [("alpha_a", grads[0], gas["alpha_a"], (0, 1, 5)), ("alpha_s", grads[1], gas["alpha_s"], (0, 2, 4))]
    for idx in [(0, 1, 5, 0), (0, 2, 5, 7), (0, 3, 4, 13), (0, 0, 5, 16)]:
        checks.append(("I", gI, I0, idx))
    for field, grad, base, idx in checks:
        gmax = float(grad.abs().max())
        h = 1e-5 * max(abs(float(base[idx])), 1e-3 * float(base.abs().max()))
        fd = (loss_with(field, idx, h) - loss_with(field, idx, -h)) / (2 * h)
        ad = float(grad[idx])
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 2e-2 * gmax), (field, idx, fd, ad)

