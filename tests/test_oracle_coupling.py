"""Pins of the oracle's implicit coupling (Sec. 2.5) and of its use in the
RK2 step: the thermal fixed point, an independent backward-Euler solve of
the static two-variable system, the equilibration closed form and ODE of
Sec. 3.6, energy bookkeeping for a moving fluid, and the quartic root
against a companion-matrix solve."""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import coupling as C
from oracle import step as S
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup

F64 = torch.float64


def box_setup(kind="mink_cart", a=0.0, level=2, n=(2, 2, 2)):
    ang = GeodesicGrid(level)
    if kind == "mink_cart":
        xf = [np.linspace(0, 1, n[d] + 1) for d in range(3)]
        bc = (("periodic", "periodic"),) * 3
    else:
        xf = [np.linspace(3.0, 4.0, n[0] + 1), np.linspace(0.8, 1.4, n[1] + 1), np.linspace(0, 0.5, n[2] + 1)]
        bc = (("outflow", "outflow"),) * 3
    return Setup(Grid(kind, a, xf, bc, 3), ang)


def gas_fields(shape, rho=1.0, u=(0.0, 0.0, 0.0), aa=0.1, a_s=0.0):
    return {"rho": torch.full(shape, rho, dtype=F64),
            "u": torch.tensor(u, dtype=F64).expand(shape + (3,)).clone(),
            "alpha_a": torch.full(shape, aa, dtype=F64),
            "alpha_s": torch.full(shape, a_s, dtype=F64), "eta": None}


@pytest.mark.parametrize("kind,a", [("mink_cart", 0.0), ("ks_sph", 0.9)])
def test_thermal_equilibrium_is_a_fixed_point(kind, a):
    st = box_setup(kind, a)
    sh = st.grid.shape
    T = torch.full(sh, 1.3, dtype=F64)
    I = (T ** 4 / (4 * math.pi))[..., None].expand(sh + (st.ang.n_ang,)).clone()
    gas = gas_fields(sh, aa=2.0, a_s=0.7)
    Ip, Tp, dR, ok = C.couple(I, T, gas, 0.05, st)
    assert ok.all()
    assert (Ip - I).abs().max() < 1e-15 * float(I.max()) * 4
    assert (Tp - T).abs().max() < 1e-14


def test_static_coupling_is_backward_euler_of_two_variable_system():
    """Static fluid, isotropic I: the update equals backward Euler of
    dE/dt = alpha (a T^4 - E), c_v dT/dt = -dE/dt, solved here by brentq."""
    st = box_setup()
    sh = st.grid.shape
    cv, aa, dt = 1.5, 0.7, 0.3
    T0, E0 = 2.0, 0.4
    I = torch.full(sh + (st.ang.n_ang,), E0 / (4 * math.pi), dtype=F64)
    Ip, Tp, _, _ = C.couple(I, torch.full(sh, T0, dtype=F64), gas_fields(sh, aa=aa), dt, st)
    # E1 = (E0 + dt alpha a T1^4) / (1 + dt alpha), cv (T1 - T0) = -(E1 - E0)
    T1 = brentq(lambda T: cv * (T - T0) + (E0 + dt * aa * T ** 4) / (1 + dt * aa) - E0, 0.0, 5.0, xtol=1e-15)
    E1 = (E0 + dt * aa * T1 ** 4) / (1 + dt * aa)
    assert abs(float(Tp[0, 0, 0]) - T1) < 1e-13
    assert abs(float((Ip[0, 0, 0] * st.ang.dOmega).sum()) - E1) < 1e-13


def test_equilibration_matches_closed_form_and_ode():
    """Sec. 3.6 set-up: Gamma = 5/3, rho = 1, p_gas = 2 (T = 2), E_rad = 1,
    alpha_a = 0.1.  T_eq solves T rho / (Gamma - 1) + T^4 = u_gas0 + u_rad0,
    and u_gas(t) follows du/dt = alpha (u0 + E0 - u - ((Gamma-1) u / rho)^4).
    The coupled RK2 steps converge to the ODE at first order and never
    overshoot T_eq."""
    st = box_setup(n=(1, 1, 1))
    sh = st.grid.shape
    gam, rho, aa = 5.0 / 3.0, 1.0, 0.1
    u0, E0 = 2.0 / (gam - 1.0), 1.0
    Teq = brentq(lambda T: T * rho / (gam - 1) + T ** 4 - (u0 + E0), 0.0, 3.0, xtol=1e-15)
    assert abs(Teq - 1.2147993409938) < 1e-12
    t_end = 10.0
    sol = solve_ivp(lambda t, u: aa * (u0 + E0 - u - ((gam - 1) * u / rho) ** 4), (0, t_end), [u0],
                    rtol=1e-12, atol=1e-14, dense_output=True)
    errs = []
    opts = S.Opts(recon="dc")
    for nsteps in (40, 80, 160):
        dt = t_end / nsteps
        I = torch.full(sh + (st.ang.n_ang,), E0 / (4 * math.pi), dtype=F64)
        T = torch.full(sh, 2.0, dtype=F64)
        prev, err = 2.0, 0.0
        for s in range(nsteps):
            I, T, src, ok = S.rk2_step(I, T, gas_fields(sh, aa=aa), dt, st, opts)
            assert ok.all()
            Tn = float(T.flatten()[0])
            assert Teq - 1e-12 <= Tn <= prev + 1e-12        # monotone, no overshoot
            prev = Tn
            E = float((I.flatten(0, 2)[0] * st.ang.dOmega).sum())
            assert abs(E + Tn * rho / (gam - 1) - (u0 + E0)) < 1e-12   # total energy
            err = max(err, abs(Tn * rho / (gam - 1) - float(sol.sol((s + 1) * dt)[0])))
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


def test_gas_source_balances_temperature_change():
    """Minkowski, static gas: the energy source -dR^0_0 equals -c_v dT."""
    st = box_setup()
    sh = st.grid.shape
    rng = np.random.default_rng(5)
    I = torch.tensor(rng.uniform(0.01, 0.2, sh + (st.ang.n_ang,)))
    T = torch.tensor(rng.uniform(0.5, 2.0, sh))
    Ip, Tp, dR, ok = C.couple(I, T, gas_fields(sh, aa=3.0, a_s=1.0), 0.1, st)
    cv = 1.5
    assert (-dR[..., 0] + cv * (Tp - T)).abs().max() < 1e-13
    # momentum change of an isotropic-source coupling of an anisotropic field
    dF = torch.einsum("...n,ni,n->...i", Ip - I, st.ang.dir, st.ang.dOmega)
    assert (dR[..., 1:] - dF).abs().max() < 1e-14


def test_moving_fluid_energy_bookkeeping():
    """Eq. coupling_tot holds exactly for a moving fluid: the fluid-frame
    energy sum of the new intensities plus c_v T is unchanged."""
    st = box_setup()
    sh = st.grid.shape
    rng = np.random.default_rng(9)
    I = torch.tensor(rng.uniform(0.01, 0.3, sh + (st.ang.n_ang,)))
    T = torch.tensor(rng.uniform(0.5, 2.0, sh))
    gas = gas_fields(sh, u=(0.3, -0.2, 0.4), aa=5.0, a_s=2.0)
    Ip, Tp, _, ok = C.couple(I, T, gas, 0.2, st)
    u = gas["u"]
    u0 = torch.sqrt(1 + (u * u).sum(-1))
    nb = u0[..., None] - torch.einsum("...i,ni->...n", u, st.ang.dir)
    Ebar = lambda X: (X * nb ** 2 * st.ang.dOmega).sum(-1)
    assert ((Ebar(Ip) + 1.5 * Tp) - (Ebar(I) + 1.5 * T)).abs().max() < 1e-13


def test_quartic_root_against_companion_matrix():
    rng = np.random.default_rng(11)
    n = 10000
    B4 = torch.tensor(10 ** rng.uniform(-6, 4, n))
    B1 = torch.tensor(10 ** rng.uniform(-4, 4, n))
    B0 = -torch.tensor(10 ** rng.uniform(-6, 4, n))
    T, ok = C.quartic_root(B4, B1, B0)
    assert ok.all()
    for i in range(0, n, 97):
        roots = np.roots([B4[i].item(), 0.0, 0.0, B1[i].item(), B0[i].item()])
        pos = [r.real for r in roots if abs(r.imag) < 1e-9 * abs(r) and r.real > 0]
        assert len(pos) == 1
        assert abs(pos[0] - float(T[i])) < 1e-9 * pos[0]
    f = B4 * T ** 4 + B1 * T + B0
    scale = B4 * T ** 4 + B1 * T + B0.abs()
    assert (f.abs() / scale).max() < 1e-14


def test_quartic_degenerate_cases():
    T, ok = C.quartic_root(torch.tensor([0.0, 2.0, 1.0]), torch.tensor([2.0, 1.0, -1.0]),
                           torch.tensor([-3.0, 0.0, -1.0]))
    assert ok.tolist() == [True, True, False]
    assert abs(float(T[0]) - 1.5) < 1e-15 and float(T[1]) == 0.0


def test_emissivity_mode_linear_solution():
    st = box_setup()
    sh = st.grid.shape
    gas = gas_fields(sh, u=(0.2, 0.0, -0.1), aa=1.5, a_s=0.8)
    gas["eta"] = torch.full(sh, 0.3, dtype=F64)
    rng = np.random.default_rng(2)
    I = torch.tensor(rng.uniform(0.01, 0.3, sh + (st.ang.n_ang,)))
    T = torch.ones(sh, dtype=F64)
    Ip, Tp, _, ok = C.couple(I, T, gas, 0.2, st, mode="emissivity")
    assert torch.equal(Tp, T)
    # the implicit equation itself holds for every bin (Eq. implicit_ii with j = eta + alpha_s E / 4pi)
    u = gas["u"]
    u0 = torch.sqrt(1 + (u * u).sum(-1))
    nb = u0[..., None] - torch.einsum("...i,ni->...n", u, st.ang.dir)
    n0 = st.nup[..., 0]
    Ebp = (Ip * nb ** 2 * st.ang.dOmega).sum(-1)
    aE = 1.5 + 0.8
    lhs = (Ip * nb ** 4) * (n0 + nb * aE * 0.2) - n0 * (I * nb ** 4)
    rhs = nb * 0.2 * (0.3 + 0.8 * Ebp[..., None] / (4 * math.pi))
    assert (lhs - rhs).abs().max() < 1e-14


def _golden(name):
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = [float(x) for x in v.split()]
    return vals


def test_static_equilibration_at_the_papers_time_resolutions():
    """The printed set-up (tests/golden/static_equilibration.txt) at 100, 10
    and 1 steps per coupling time: every run heads to T_eq without
    overshooting and conserves gas + radiation energy; finer steps end
    closer to T_eq after the same time."""
    g = _golden("static_equilibration.txt")
    gam, rho, aa = g["gamma"][0], g["rho"][0], g["alpha_a"][0]
    T0 = g["p_gas0"][0] / rho                    # p = rho T in these units
    u0, E0 = T0 * rho / (gam - 1.0), g["u_rad0"][0]
    Teq = brentq(lambda T: T * rho / (gam - 1) + T ** 4 - (u0 + E0), 0.0, 3.0, xtol=1e-15)
    st = box_setup(n=(1, 1, 1))
    sh = st.grid.shape
    t_end = 5.0 / aa
    gaps = []
    for per in g["steps_per_coupling_time"]:
        dt = 1.0 / (aa * per)
        I = torch.full(sh + (st.ang.n_ang,), E0 / (4 * math.pi), dtype=F64)
        T = torch.full(sh, T0, dtype=F64)
        prev = T0
        for _ in range(int(round(t_end / dt))):
            I, T, src, ok = S.rk2_step(I, T, gas_fields(sh, aa=aa, rho=rho), dt, st,
                                       S.Opts(recon="dc", gamma=gam))
            assert ok.all()
            Tn = float(T.flatten()[0])
            assert Teq - 1e-12 <= Tn <= prev + 1e-12          # monotone towards T_eq, no overshoot
            E = float((I.flatten(0, 2)[0] * st.ang.dOmega).sum())
            assert abs(E + Tn * rho / (gam - 1) - (u0 + E0)) < 1e-12 * (u0 + E0)
            prev = Tn
        gaps.append(prev - Teq)
    assert gaps[0] < gaps[1] < gaps[2]
    assert gaps[2] < 0.1 * (T0 - Teq)                          # even one step per coupling time gets close


def _gas_from_conserved(D, E, Sx, gam):
    """(rho, p, u^1) of an ideal gas from rho u^0, w u^0 u^0 - p and w u^0 u^1."""
    def resid(u1):
        u0 = math.sqrt(1.0 + u1 * u1)
        w = Sx / (u0 * u1)
        rho = D / u0
        p = (w - rho) * (gam - 1.0) / gam
        return w * u0 * u0 - p - E
    u1 = brentq(resid, 1e-12, 50.0, xtol=1e-15, rtol=1e-15)
    u0 = math.sqrt(1.0 + u1 * u1)
    w = Sx / (u0 * u1)
    rho = D / u0
    return rho, (w - rho) * (gam - 1.0) / gam, u1


def test_moving_equilibration_follows_the_papers_ode():
    """Sec. 3 "Equilibration", moving case (Eq. moving_equilibration): the
    static set-up with initial u^1 = 1.  The coupled RK2 steps, with the gas
    energy-momentum advanced by the returned source (-dR^0_mu) and the gas
    state recovered from rho u^0, w u^0 u^0 - p, w u^0 u^1 after each step,
    converge at first order in dt to the ODE system the paper prints for the
    same angle bins; total energy and momentum are conserved."""
    from scipy.integrate import solve_ivp
    g = _golden("static_equilibration.txt")
    gam, rho0, aa = g["gamma"][0], g["rho"][0], g["alpha_a"][0]
    p0, E0, u10 = g["p_gas0"][0], g["u_rad0"][0], 1.0
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

    t_end = 20.0
    sol = solve_ivp(rhs, (0, t_end), np.concatenate([[Eg0, S0], I0]), rtol=1e-11, atol=1e-13, dense_output=True)
    errs = []
    for nsteps in (25, 50, 100):
        dt = t_end / nsteps
        I = torch.tensor(np.broadcast_to(I0, sh + (len(dO),)).copy())
        Eg, Sx = Eg0, S0
        rho, p, u1 = rho0, p0, u10
        err = 0.0
        for s in range(nsteps):
            gas = gas_fields(sh, rho=rho, u=(u1, 0.0, 0.0), aa=aa)
            T = torch.full(sh, p / rho, dtype=F64)
            I, Tn, src, ok = S.rk2_step(I, T, gas, dt, st, S.Opts(recon="dc", gamma=gam))
            assert ok.all()
            Eg, Sx = Eg - float(src.flatten()[0]), Sx + float(src.flatten()[1])
            rho, p, u1 = _gas_from_conserved(D, Eg, Sx, gam)
            Ir = I.flatten(0, 2)[0].numpy()
            # conservation of total energy and x-momentum
            assert abs(Eg + (Ir * dO).sum() - (Eg0 + E0)) < 1e-11 * (Eg0 + E0)
            assert abs(Sx + (Ir * n1 * dO).sum() - S0) < 1e-11 * S0
            ref = sol.sol((s + 1) * dt)
            err = max(err, abs(Eg - ref[0]) / ref[0], abs(Sx - ref[1]) / ref[1])
        errs.append(err)
    assert errs[2] < 1e-2
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6
