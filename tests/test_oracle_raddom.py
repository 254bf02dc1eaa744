"""Pins of the oracle's radiation-dominated velocity substitution (end of
Sec. 2.5): inactive below the trigger, the fraction of a static gas in
closed form, the radiation velocity under strong coupling, symmetry under a
rotation by pi about the 2-axis, and first-order convergence to the paper's
moving-equilibration ODE (Eq. moving_equilibration) in a radiation-dominated
set-up where the substitution is active.

The closed form: for a gas at rest (u = (1, 0, 0, 0)) the force is
G^a = alpha_E R^{0a}, the gas momentum T_gas^{0a} = 0 and
T_rad^{0a} = w gamma^2 v^a with v^a = R^{0a} / R^{00}, so every component
has the same fraction f = alpha_E R^{00} dt (1 - v^2) / w."""
import math

import numpy as np
import torch

from oracle import coupling as C
from oracle import step as S
from tests.test_oracle_coupling import _gas_from_conserved, box_setup, gas_fields

F64 = torch.float64


def _aniso_I(st, E, a):
    """I = E/(4 pi) (1 + a . n): R^{00} = E, R^{0a} = E a / 3 (to roundoff)."""
    n = st.ang.dir
    base = E / (4 * math.pi) * (1.0 + n @ torch.tensor(a, dtype=F64))
    return base.expand(st.grid.shape + (st.ang.n_ang,)).clone()


def _moments(I, st):
    dO, n = st.ang.dOmega, st.ang.dir
    return (I * dO).sum(-1), torch.einsum("...n,na,n->...a", I, n, dO)


def test_inactive_below_the_trigger_is_the_plain_coupling():
    """E_bar < rho + u_gas: the substitution leaves the coupling untouched
    (bit for bit)."""
    st = box_setup(n=(2, 1, 1))
    sh = st.grid.shape
    I = _aniso_I(st, 0.5, (0.3, -0.2, 0.1))
    T = torch.full(sh, 1.0, dtype=F64)
    gas = gas_fields(sh, rho=1.0, u=(0.2, -0.1, 0.05), aa=0.3, a_s=0.2)
    u_sub, f, act = C.substituted_velocity(I, T, gas, 0.1, st)
    assert not act.any()
    plain = C.couple(I, T, gas, 0.1, st)
    sub = C.couple(I, T, gas, 0.1, st, rad_dom=True)
    for p, q in zip(plain, sub):
        assert torch.equal(p, q)


def test_static_gas_fraction_closed_form():
    st = box_setup(n=(1, 1, 1), level=3)
    sh = st.grid.shape
    E, rho, T0, aa, a_s, dt, gam = 1.0, 1e-3, 1.0, 0.05, 0.02, 0.01, 5.0 / 3.0
    I = _aniso_I(st, E, (0.3, -0.2, 0.1))
    T = torch.full(sh, T0, dtype=F64)
    gas = gas_fields(sh, rho=rho, u=(0.0, 0.0, 0.0), aa=aa, a_s=a_s)
    u_sub, f, act = C.substituted_velocity(I, T, gas, dt, st)
    assert act.all()
    R00, R0a = _moments(I, st)
    v = R0a / R00[..., None]
    v2 = (v * v).sum(-1)
    w = rho + gam / (gam - 1.0) * rho * T0
    f_ref = (aa + a_s) * R00 * dt * (1.0 - v2) / w
    assert 0.1 < float(f_ref.min()) and float(f_ref.max()) < 0.9        # the clamp is not engaged
    assert float((f - f_ref[..., None]).abs().max()) < 1e-13
    u_ref = f_ref[..., None] * v / torch.sqrt(1.0 - v2)[..., None]
    assert float((u_sub - u_ref).abs().max()) < 1e-15


def test_strong_coupling_selects_the_radiation_velocity():
    """alpha_E dt large: f^1 clamps to 1, the coupling runs at the radiation
    velocity, and equals the plain coupling of a gas given that velocity."""
    st = box_setup(n=(1, 1, 1), level=3)
    sh = st.grid.shape
    I = _aniso_I(st, 2.0, (0.9, 0.0, 0.0))
    T = torch.full(sh, 0.8, dtype=F64)
    gas = gas_fields(sh, rho=1e-2, u=(0.05, 0.0, 0.0), aa=20.0, a_s=5.0)
    dt = 0.5
    u_sub, f, act = C.substituted_velocity(I, T, gas, dt, st)
    assert act.all()
    R00, R0a = _moments(I, st)
    v = R0a / R00[..., None]
    u_rad = v / torch.sqrt(1.0 - (v * v).sum(-1))[..., None]
    assert float(f[..., 0].min()) == 1.0
    assert float((u_sub - u_rad).abs().max()) < 1e-14
    g2 = dict(gas)
    g2["u"] = u_rad
    sub = C.couple(I, T, gas, dt, st, rad_dom=True)
    plain = C.couple(I, T, g2, dt, st)
    for p, q in zip(sub[:3], plain[:3]):
        assert float((p - q).abs().max()) <= 1e-13 * float(q.abs().max())


def test_substitution_commutes_with_a_rotation_by_pi_about_the_2_axis():
    """(x, y, z) -> (-x, y, -z) maps bins by the grid's own symmetry; the
    per-component fractions and the coupling transform with it."""
    st = box_setup(n=(1, 1, 1), level=3)
    sh = st.grid.shape
    perm = st.ang.perm_pi2
    I = _aniso_I(st, 1.5, (0.4, -0.3, 0.25))
    T = torch.full(sh, 0.9, dtype=F64)
    gas = gas_fields(sh, rho=2e-2, u=(0.15, 0.12, 0.2), aa=0.4, a_s=0.3)
    sgn = torch.tensor([-1.0, 1.0, -1.0], dtype=F64)
    gr = dict(gas)
    gr["u"] = gas["u"] * sgn
    Ir = I[..., perm]
    dt = 0.02
    u1, f1, a1 = C.substituted_velocity(I, T, gas, dt, st)
    u2, f2, a2 = C.substituted_velocity(Ir, T, gr, dt, st)
    assert a1.all() and a2.all()
    assert float(f1.min()) > 0.0 and float(f1.max()) < 1.0
    assert float((u2 - u1 * sgn).abs().max()) < 1e-14
    assert float((f2 - f1).abs().max()) < 1e-12
    Ip1, Tp1, dR1, _ = C.couple(I, T, gas, dt, st, rad_dom=True)
    Ip2, Tp2, dR2, _ = C.couple(Ir, T, gr, dt, st, rad_dom=True)
    assert float((Ip2 - Ip1[..., perm]).abs().max()) < 1e-13 * float(Ip1.abs().max())
    assert float((Tp2 - Tp1).abs().max()) < 1e-13
    # Minkowski Cartesian: the coordinate frame is the tetrad frame
    s4 = torch.tensor([1.0, -1.0, 1.0, -1.0], dtype=F64)
    assert float((dR2 - dR1 * s4).abs().max()) < 1e-13 * float(dR1.abs().max())


def test_radiation_dominated_moving_equilibration_converges_to_the_ode():
    """The moving equilibration of Sec. 3 with a radiation energy ten times
    the gas inertia (E_rad = 40, rho = 1, p = 2): the substitution is active,
    the coupled steps with the gas advanced by the returned source converge
    at first order in dt to the paper's ODE system, energy and momentum are
    conserved, and at every dt the error is below that of the same steps
    without the substitution (the frozen velocity is what the substitution
    corrects when radiation dominates)."""
    from scipy.integrate import solve_ivp
    gam, rho0, aa, p0, E0, u10 = 5.0 / 3.0, 1.0, 0.1, 2.0, 40.0, 1.0
    st = box_setup(n=(1, 1, 1))
    sh = st.grid.shape
    dirs, dO = st.ang.dir.numpy(), st.ang.dOmega.numpy()
    n1 = dirs[:, 0]
    u00 = math.sqrt(1 + u10 ** 2)
    D = rho0 * u00
    w0 = rho0 + gam / (gam - 1) * p0
    Eg0, S0 = w0 * u00 * u00 - p0, w0 * u00 * u10
    I0 = np.full(len(dO), E0 / (4 * math.pi))

    def rhs(t, y):
        Eg, Sx, I = y[0], y[1], y[2:]
        rho, p, u1 = _gas_from_conserved(D, Eg, Sx, gam)
        u0 = math.sqrt(1 + u1 * u1)
        T4 = (p / rho) ** 4
        R00, R01, R11 = (I * dO).sum(), (I * n1 * dO).sum(), (I * n1 * n1 * dO).sum()
        nb = u0 - u1 * n1
        return np.concatenate([[aa * (u0 * R00 - u1 * R01 - T4 * u0), aa * (u0 * R01 - u1 * R11 - T4 * u1)],
                               aa * (T4 / (4 * math.pi) * nb ** -3 - nb * I)])

    t_end = 10.0
    sol = solve_ivp(rhs, (0, t_end), np.concatenate([[Eg0, S0], I0]), rtol=1e-11, atol=1e-13, dense_output=True)

    def run(nsteps, rad_dom):
        dt = t_end / nsteps
        I = torch.tensor(np.broadcast_to(I0, sh + (len(dO),)).copy())
        Eg, Sx = Eg0, S0
        rho, p, u1 = rho0, p0, u10
        err, active = 0.0, 0
        for s in range(nsteps):
            gas = gas_fields(sh, rho=rho, u=(u1, 0.0, 0.0), aa=aa)
            T = torch.full(sh, p / rho, dtype=F64)
            active += int(C.substituted_velocity(I, T, gas, dt, st)[2].all())
            I, Tn, src, ok = S.rk2_step(I, T, gas, dt, st, S.Opts(recon="dc", gamma=gam, rad_dom=rad_dom))
            assert ok.all()
            Eg, Sx = Eg - float(src.flatten()[0]), Sx + float(src.flatten()[1])
            rho, p, u1 = _gas_from_conserved(D, Eg, Sx, gam)
            Ir = I.flatten(0, 2)[0].numpy()
            assert abs(Eg + (Ir * dO).sum() - (Eg0 + E0)) < 1e-11 * (Eg0 + E0)
            assert abs(Sx + (Ir * n1 * dO).sum() - S0) < 1e-11 * S0
            ref = sol.sol((s + 1) * dt)
            err = max(err, abs(Eg - ref[0]) / ref[0], abs(Sx - ref[1]) / ref[1])
        return err, active

    errs = []
    for nsteps in (25, 50, 100):
        err, active = run(nsteps, True)
        assert active == nsteps
        errs.append(err)
        assert err < 0.85 * run(nsteps, False)[0]
    assert errs[2] < 0.08
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6


def test_substituted_coupling_gradient_matches_finite_differences():
    """The oracle's reverse-mode gradient of one step with the substitution
    (the reference the GPU adjoint is compared with) against central
    differences in alpha_a, alpha_s, T^0 and intensities, at cells where the
    substitution is active with momentum fractions strictly inside (0, 1)
    (so the velocity depends smoothly on the inputs), on a flat moving-gas
    block with the density spread over 1e-3 .. 10.  Steps of 1e-4 relative
    (at 1e-5 roundoff dominates the small opacities' differences)."""
    import workloads as W
    from oracle import adjoint as A
    from oracle.angles import GeodesicGrid
    from oracle.transport import Grid, Setup
    w = W.make("turb3d", n=(5, 4, 3), level=1)
    w["rho"] = 10.0 ** np.random.default_rng(4).uniform(-3, 1, w["T"].shape)
    st = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), GeodesicGrid(1))
    gas = {k: torch.tensor(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s")}
    gas["eta"] = None
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    dt = 0.004
    o = S.Opts(recon="plm", rad_dom=True)
    u_sub, f, act = C.substituted_velocity(I0, T0, gas, dt, st)
    interior = act & ((f > 1e-6) & (f < 1 - 1e-6)).all(-1)
    assert int(interior.sum()) >= 4 and int((~act).sum()) >= 4
    rng = np.random.default_rng(8)
    lam, lamT = torch.tensor(rng.normal(size=I0.shape)), torch.tensor(rng.normal(size=T0.shape))

    def obj(I, T, g):
        I2, T2, _, ok = S.rk2_step(I, T, g, dt, st, o)
        assert bool(ok.all())
        return float((I2 * lam).sum() + (T2 * lamT).sum())

    lI, lT, ga, gs, _ = A.step_vjp(I0, T0, gas, dt, st, o, lam, lamT)
    cells = [tuple(c) for c in interior.nonzero().tolist()[:4]]
    for c in cells:
        for key, grad in (("alpha_a", ga), ("alpha_s", gs)):
            h = 1e-4 * float(gas[key][c])
            gp, gm = dict(gas), dict(gas)
            gp[key] = gas[key].clone()
            gp[key][c] += h
            gm[key] = gas[key].clone()
            gm[key][c] -= h
            fd = (obj(I0, T0, gp) - obj(I0, T0, gm)) / (2 * h)
            assert abs(fd - float(grad[c])) <= 1e-6 * max(abs(fd), 1e-3 * float(grad.abs().max())), (key, c)
        h = 1e-4 * float(T0[c])
        Tp, Tm = T0.clone(), T0.clone()
        Tp[c] += h
        Tm[c] -= h
        fd = (obj(I0, Tp, gas) - obj(I0, Tm, gas)) / (2 * h)
        assert abs(fd - float(lT[c])) <= 1e-6 * max(abs(fd), 1e-3 * float(lT.abs().max())), ("T", c)
        for n in (0, 5):
            h = 1e-4 * float(I0[c + (n,)])
            Ip, Im = I0.clone(), I0.clone()
            Ip[c + (n,)] += h
            Im[c + (n,)] -= h
            fd = (obj(Ip, T0, gas) - obj(Im, T0, gas)) / (2 * h)
            assert abs(fd - float(lI[c + (n,)])) <= 1e-6 * max(abs(fd), 1e-3 * float(lI.abs().max())), ("I", c, n)
