"""Pins of the oracle's multigroup transport (Sec. 2.2, Eq.
radiation_integral_frequency) against facts fixed outside it:

* one group spanning all frequencies is the gray step, bit for bit;
* the frequency fluxes telescope: with nothing crossing nu = 0 and
  nu = infinity, the sum over groups of a linear multigroup step (donor
  cell, no coupling or fixed emissivity with group-independent opacities)
  is the gray step of the summed intensity;
* the frequency symbol: omega^0hat vanishes for static observers of flat
  space; for static observers of Schwarzschild it is the gravitational
  redshift, d ln nu / dt = -n^rhat / r^2, i.e. omega^0hat_{AB} n^A n^B =
  n^rhat / (r^2 (1 - 2/r)^(1/2)), whose integral along a radial ray is the
  (1 - 2M/r)^(1/2) factor; in Kerr-Schild, n^nu equals the rate of change of
  the normal observer's frequency along a null geodesic integrated with its
  own Christoffel symbols;
* the donor-cell edge fluxes, expanded by hand for three groups.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import frequency as FQ
from oracle import geometry as G
from oracle import step as OS
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup

F64 = torch.float64
INF = float("inf")


def _setup(w, level):
    return Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), GeodesicGrid(level))


def _groups(w, G_, rng, same_opacity=False):
    sh = w["T"].shape
    gas = {"rho": torch.tensor(w["rho"]), "u": torch.tensor(w["u"])}
    if same_opacity:
        gas["alpha_a"] = torch.tensor(np.broadcast_to(w["alpha_a"], (G_,) + sh).copy())
        gas["alpha_s"] = torch.tensor(np.broadcast_to(w["alpha_s"], (G_,) + sh).copy())
    else:
        gas["alpha_a"] = torch.tensor(w["alpha_a"][None] * rng.uniform(0.5, 2.0, (G_,) + sh))
        gas["alpha_s"] = torch.tensor(w["alpha_s"][None] * rng.uniform(0.5, 2.0, (G_,) + sh))
    gas["eta"] = torch.tensor(rng.uniform(0.01, 0.1, (G_,) + sh))
    return gas


def test_one_group_is_the_gray_step():
    w = W.make("torus3d", n=(5, 4, 4), level=2)
    st = _setup(w, 2)
    rng = np.random.default_rng(1)
    gas = _groups(w, 1, rng)
    I0 = torch.tensor(w["I0"])[None]
    T = torch.tensor(w["T"])
    for couple in (True, False):
        o = OS.Opts(mode="emissivity", couple=couple)
        a, _, sa, ok = FQ.rk2_step_groups(I0, T, gas, 1e-3, st, o, [0.0, INF])
        g1 = {"rho": gas["rho"], "u": gas["u"], "alpha_a": gas["alpha_a"][0], "alpha_s": gas["alpha_s"][0],
              "eta": gas["eta"][0]}
        b, _, sb, okb = OS.rk2_step(I0[0], T, g1, 1e-3, st, o)
        assert bool(ok.all()) and bool(okb.all())
        assert torch.equal(a[0], b) and torch.equal(sa[0], sb)


@pytest.mark.parametrize("couple", [False, True])
def test_frequency_fluxes_telescope(couple):
    """Kerr-Schild (omega^0hat != 0) with a moving gas: the sum over groups
    equals the gray step of the sum (donor cell in space and angle, so the
    step is linear in I)."""
    w = W.make("torus3d_big", n=(5, 4, 4), level=2)
    st = _setup(w, 2)
    assert float(FQ.omega0_nn(st).abs().max()) > 1e-3
    rng = np.random.default_rng(2)
    edges = [0.0, 0.5, 1.0, 2.0, 4.0, INF]
    Gn = len(edges) - 1
    gas = _groups(w, Gn, rng, same_opacity=True)
    I0 = torch.tensor(rng.uniform(0.2, 1.0, (Gn,) + w["I0"].shape))
    T = torch.tensor(w["T"])
    o = OS.Opts(recon="dc", recon_ang="dc", mode="emissivity", couple=couple)
    dt = 2e-3
    Ig, _, srcg, ok = FQ.rk2_step_groups(I0, T, gas, dt, st, o, edges)
    assert bool(ok.all())
    # the frequency fluxes move energy between groups: the groups differ from a gray step of each
    assert float((FQ.frequency_divergence(I0, st, edges)).abs().max()) > 1e-3 * float(I0.abs().max())
    g1 = {"rho": gas["rho"], "u": gas["u"], "alpha_a": gas["alpha_a"][0], "alpha_s": gas["alpha_s"][0],
          "eta": gas["eta"].sum(0)}
    Ib, _, srcb, okb = OS.rk2_step(I0.sum(0), T, g1, dt, st, o)
    assert float((Ig.sum(0) - Ib).abs().max()) < 1e-14 * float(Ib.abs().max())
    assert float((srcg.sum(0) - srcb).abs().max()) < 1e-13 * float(srcb.abs().max() + Ib.abs().max())


def test_frequency_symbol_vanishes_for_static_flat_observers():
    for name, kind in (("turb3d", "mink_cart"), ("torus3d", "mink_sph")):
        w = W.make(name, n=(4, 4, 4), level=1, with_intensity=False)
        w["kind"], w["spin"] = kind, 0.0
        if kind == "mink_sph":
            w["xf"][0] = np.linspace(2.0, 5.0, 5)
        st = _setup(w, 2)
        assert float(FQ.omega0_nn(st).abs().max()) < 1e-15


def test_schwarzschild_static_observer_redshift():
    """omega^0hat_{AB} n^A n^B = n^rhat / (r^2 sqrt(1 - 2/r)) (n^rhat = the
    bin's 2hat component): integrating d ln nu = -n^rhat dr / (r^2 (1 - 2/r))
    along an outgoing radial ray (dr/dt = (1 - 2/r) n^rhat) from r_e to r_o
    gives nu_o / nu_e = sqrt((1 - 2/r_e) / (1 - 2/r_o))."""
    ang = GeodesicGrid(3)
    xf = [np.linspace(3.0, 12.0, 6), np.linspace(0.3, 2.8, 5), np.linspace(0.0, 1.0, 3)]
    st = Setup(Grid("schw_sph", 0.0, xf, (("outflow", "outflow"),) * 3, 3), ang)
    q = FQ.omega0_nn(st)
    r = st.grid.centres()[..., 0]
    want = ang.dir[:, 1] / (r ** 2 * torch.sqrt(1.0 - 2.0 / r))[..., None]
    assert float((q - want).abs().max()) < 1e-13
    # the integral along a radial ray reproduces the static redshift factor
    re, ro = 3.0, 12.0
    rr = np.linspace(re, ro, 20001)
    dlnnu = -1.0 / (rr ** 2 * (1.0 - 2.0 / rr))            # d ln nu / dr = (-q / n^0) / (dr/dt) at n^rhat = 1
    integral = np.sum(0.5 * (dlnnu[1:] + dlnnu[:-1]) * np.diff(rr))
    assert abs(math.exp(integral) - math.sqrt((1 - 2 / re) / (1 - 2 / ro))) < 1e-8


def _christoffel_fd(kind, a, x, h=1e-5):
    g = G.metric(kind, a, x)
    dg = torch.zeros(4, 4, 4, dtype=F64)
    for d in range(3):
        dx = torch.zeros(3, dtype=F64)
        dx[d] = h
        dg[:, :, d + 1] = (G.metric(kind, a, x + dx) - G.metric(kind, a, x - dx)) / (2 * h)
    low = torch.zeros(4, 4, 4, dtype=F64)
    for k in range(4):
        for d in range(4):
            for s in range(4):
                low[k, d, s] = 0.5 * (dg[k, s, d] + dg[k, d, s] - dg[d, s, k])
    return torch.einsum("ek,kds->eds", torch.linalg.inv(g), low)


@pytest.mark.parametrize("kind,a,p,n", [
    ("ks_sph", 0.9, (4.0, 1.0, 0.3), (0.3, -0.5, 0.81)),
    ("ks_sph", 0.9, (2.5, 2.0, 1.3), (-0.7, 0.1, 0.2)),
    ("ks_sph", 0.5, (6.0, 1.6, 0.0), (0.0, 1.0, 0.0)),
    ("schw_sph", 0.0, (5.0, 1.2, 0.4), (0.2, 0.9, -0.3)),
])
def test_frequency_symbol_matches_geodesic(kind, a, p, n):
    """A null geodesic with k = e (1, nhat) at lambda = 0 (tetrad frequency 1)
    is integrated both ways (RK4, Christoffels by finite differences of the
    metric); d k^0hat / d lambda must equal n^nu / nu = -omega^0hat_{AB} n^A n^B."""
    x = torch.tensor((0.0,) + p, dtype=F64)
    nhat = torch.tensor(n, dtype=F64)
    nhat = nhat / nhat.norm()
    e = G.tetrad(kind, a, x[1:])
    k = e @ torch.cat([torch.ones(1, dtype=F64), nhat])
    h, steps = 1e-3, 4

    def rhs(y):
        gam = _christoffel_fd(kind, a, y[1:4])
        return torch.cat([y[4:], -torch.einsum("mab,a,b->m", gam, y[4:], y[4:])])

    def nu_after(sign):
        y = torch.cat([x, k])
        for _ in range(steps):
            k1 = rhs(y)
            k2 = rhs(y + 0.5 * sign * h * k1)
            k3 = rhs(y + 0.5 * sign * h * k2)
            k4 = rhs(y + sign * h * k3)
            y = y + sign * h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        return float(torch.linalg.solve(G.tetrad(kind, a, y[1:4]), y[4:])[0])

    dnu = (nu_after(+1) - nu_after(-1)) / (2 * h * steps)
    w = G.ricci_rotation(kind, a, x[1:])
    n4 = torch.cat([torch.ones(1, dtype=F64), nhat])
    q0 = float(torch.einsum("AB,A,B->", w[0], n4, n4))
    assert abs(dnu - (-q0)) < 2e-6 * max(1.0, abs(q0))
    if kind == "ks_sph" and p[0] < 5:
        assert abs(q0) > 1e-2           # a non-trivial rate is being checked


def test_donor_cell_edge_fluxes_by_hand():
    """Three groups with edges (0.5, 1, 2, 4): at every cell and bin the edge
    fluxes are nu_f s n_0 times the upwind group's mean specific intensity
    (lower group for s > 0, upper for s < 0), nothing enters from outside."""
    w = W.make("torus3d", n=(3, 3, 2), level=1)
    st = _setup(w, 1)
    rng = np.random.default_rng(5)
    edges = [0.5, 1.0, 2.0, 4.0]
    Ig = torch.tensor(rng.uniform(0.1, 1.0, (3,) + w["I0"].shape))
    D = FQ.frequency_divergence(Ig, st, edges).numpy()
    q = FQ.omega0_nn(st).numpy()
    n0 = st.nlow[..., 0].numpy()
    I = Ig.numpy()
    dnu = [0.5, 1.0, 2.0]
    for idx in np.ndindex(q.shape):
        s = -q[idx]
        m = [I[(g,) + idx] / dnu[g] for g in range(3)]
        F = [0.0] * 4
        F[0] = 0.5 * s * n0[idx] * m[0] if s < 0 else 0.0
        F[1] = 1.0 * s * n0[idx] * (m[0] if s > 0 else m[1])
        F[2] = 2.0 * s * n0[idx] * (m[1] if s > 0 else m[2])
        F[3] = 4.0 * s * n0[idx] * m[2] if s > 0 else 0.0
        for g in range(3):
            assert abs(D[(g,) + idx] - (F[g + 1] - F[g])) <= 1e-15 * max(1.0, abs(F[g + 1]) + abs(F[g]))
