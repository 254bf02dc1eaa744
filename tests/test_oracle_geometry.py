"""Pins of the oracle's metric, tetrad and Ricci rotation coefficients
(Secs. 2.1-2.2, Eq. tetrad, Eq. ricci) against textbook closed forms, an
independent null-geodesic integration and the Kerr circular photon orbits
(Sec. 3.3, the orbit radii r_pm)."""
import math

import numpy as np
import pytest
import torch

from oracle import geometry as G

PTS = [(3.1, 1.1, 0.2), (1.7, 0.4, 2.0), (12.0, 2.9, 5.5), (2.2, math.pi / 2, 1.0)]


def _x(p):
    return torch.tensor(p, dtype=torch.float64)


def ks_inverse(r, th, a):
    """Kerr-Schild inverse metric (standard closed form, M = 1)."""
    sig = r * r + a * a * math.cos(th) ** 2
    delta = r * r - 2 * r + a * a
    gi = np.zeros((4, 4))
    gi[0, 0] = -(1 + 2 * r / sig)
    gi[0, 1] = gi[1, 0] = 2 * r / sig
    gi[1, 1] = delta / sig
    gi[1, 3] = gi[3, 1] = a / sig
    gi[2, 2] = 1 / sig
    gi[3, 3] = 1 / (sig * math.sin(th) ** 2)
    return gi


@pytest.mark.parametrize("kind,a", [("mink_cart", 0.0), ("mink_sph", 0.0), ("ks_sph", 0.9), ("ks_sph", 0.5)])
def test_tetrad_orthonormal_and_normal(kind, a):
    for p in PTS:
        x = _x(p)
        g, e = G.metric(kind, a, x), G.tetrad(kind, a, x)
        assert (e.T @ g @ e - G.ETA).abs().max() < 1e-13
        # spatial legs have no time component; e_0 is the normal observer
        assert e[0, 1:].abs().max() == 0.0
        if kind == "ks_sph":
            gi = torch.tensor(ks_inverse(p[0], p[1], a))
            lapse = (-gi[0, 0]) ** -0.5
            assert (e[:, 0] + lapse * gi[0, :]).abs().max() < 1e-13
        # right-handed spatial triad: det of the tetrad matches sqrt(-g)
        assert float(torch.linalg.det(e)) * float(torch.sqrt(-torch.linalg.det(g))) > 0


def test_ks_inverse_and_volume_element():
    a = 0.9
    for p in PTS:
        x = _x(p)
        g = G.metric("ks_sph", a, x)
        gi = torch.tensor(ks_inverse(p[0], p[1], a))
        assert (g @ gi - torch.eye(4, dtype=torch.float64)).abs().max() < 1e-13
        sig = p[0] ** 2 + a * a * math.cos(p[1]) ** 2
        assert abs(math.sqrt(-float(torch.linalg.det(g))) - sig * math.sin(p[1])) < 1e-12 * sig


def test_exact_volumes_match_quadrature():
    """Delta V and Delta A against Gauss-Legendre quadrature of sqrt(-det g)."""
    from numpy.polynomial.legendre import leggauss
    xg, wg = leggauss(12)
    a = 0.9
    lo, hi = np.array([2.0, 0.3, 0.1]), np.array([2.6, 0.7, 0.5])

    def sqrtg(r, th):
        return math.sqrt(-float(torch.linalg.det(G.metric("ks_sph", a, _x((r, th, 0.0))))))

    def nodes(l, h):
        return 0.5 * (h - l) * xg + 0.5 * (h + l), 0.5 * (h - l) * wg

    rr, wr = nodes(lo[0], hi[0])
    tt, wt = nodes(lo[1], hi[1])
    V = sum(wr[i] * wt[j] * sqrtg(rr[i], tt[j]) for i in range(12) for j in range(12)) * (hi[2] - lo[2])
    Vx = float(G.cell_volume("ks_sph", a, torch.tensor(lo), torch.tensor(hi)))
    assert abs(V - Vx) < 1e-12 * V
    Ar = sum(wt[j] * sqrtg(lo[0], tt[j]) for j in range(12)) * (hi[2] - lo[2])
    assert abs(Ar - float(G.face_area("ks_sph", a, 0, torch.tensor(lo), torch.tensor(hi)))) < 1e-12 * Ar
    At = sum(wr[i] * sqrtg(rr[i], lo[1]) for i in range(12)) * (hi[2] - lo[2])
    assert abs(At - float(G.face_area("ks_sph", a, 1, torch.tensor(lo), torch.tensor(hi)))) < 1e-12 * At
    Ap = sum(wr[i] * wt[j] * sqrtg(rr[i], tt[j]) for i in range(12) for j in range(12))
    assert abs(Ap - float(G.face_area("ks_sph", a, 2, torch.tensor(lo), torch.tensor(hi)))) < 1e-12 * Ap


def test_cartesian_minkowski_has_no_rotation():
    for p in PTS:
        assert G.ricci_rotation("mink_cart", 0.0, _x(p)).abs().max() == 0.0


def test_flat_spherical_closed_form():
    """Orthonormal spherical triad (1=phi, 2=r, 3=theta): nabla_theta r = theta/r,
    nabla_theta theta = -r/r, nabla_phi r = phi/r, nabla_phi theta = cot phi/r,
    nabla_phi phi = -(r + cot theta)/r; all others vanish."""
    for (r, th, ph) in PTS:
        w = G.ricci_rotation("mink_sph", 0.0, _x((r, th, ph)))
        ref = torch.zeros(4, 4, 4, dtype=torch.float64)
        cot = math.cos(th) / math.sin(th)
        ref[3, 2, 3] = 1 / r
        ref[2, 3, 3] = -1 / r
        ref[1, 2, 1] = 1 / r
        ref[1, 3, 1] = cot / r
        ref[2, 1, 1] = -1 / r
        ref[3, 1, 1] = -cot / r
        assert (w - ref).abs().max() < 1e-14 * max(1, abs(cot))


@pytest.mark.parametrize("kind,a", [("mink_sph", 0.0), ("ks_sph", 0.9)])
def test_rotation_coefficients_antisymmetric(kind, a):
    for p in PTS:
        w = G.ricci_rotation(kind, a, _x(p))
        wl = torch.einsum("CD,DAB->CAB", G.ETA, w)
        assert (wl + wl.transpose(0, 1)).abs().max() < 1e-13


def test_rotation_coefficients_match_finite_differences():
    """omega from central differences of the tetrad and metric (h = 1e-5)."""
    a, h = 0.9, 1e-5
    x = _x((3.1, 1.1, 0.2))
    e = G.tetrad("ks_sph", a, x)
    g = G.metric("ks_sph", a, x)
    de = torch.zeros(4, 4, 4, dtype=torch.float64)
    dg = torch.zeros(4, 4, 4, dtype=torch.float64)
    for d in range(3):
        dx = torch.zeros(3, dtype=torch.float64)
        dx[d] = h
        de[:, :, d + 1] = (G.tetrad("ks_sph", a, x + dx) - G.tetrad("ks_sph", a, x - dx)) / (2 * h)
        dg[:, :, d + 1] = (G.metric("ks_sph", a, x + dx) - G.metric("ks_sph", a, x - dx)) / (2 * h)
    gi = torch.linalg.inv(g)
    low = torch.zeros(4, 4, 4, dtype=torch.float64)
    for k in range(4):
        for d in range(4):
            for s in range(4):
                low[k, d, s] = 0.5 * (dg[k, s, d] + dg[k, d, s] - dg[d, s, k])
    gam = torch.einsum("ek,kds->eds", gi, low)
    einv = torch.linalg.inv(e)
    w = torch.zeros(4, 4, 4, dtype=torch.float64)
    for C in range(4):
        for A in range(4):
            for B in range(4):
                acc = 0.0
                for eps in range(4):
                    for dl in range(4):
                        cov = de[eps, A, dl] + sum(gam[eps, dl, s] * e[s, A] for s in range(4))
                        acc += einv[C, eps] * e[dl, B] * cov
                w[C, A, B] = acc
    assert (w - G.ricci_rotation("ks_sph", a, x)).abs().max() < 1e-8


def _angular_velocity(kind, a, x, nhat):
    """V = -(Q_vec - nhat Q^0), Q^C = omega^C_AB n^A n^B: d nhat / d lambda (nu = 1)."""
    w = G.ricci_rotation(kind, a, x)
    n4 = torch.cat([torch.ones(1, dtype=torch.float64), nhat])
    Q = torch.einsum("CAB,A,B->C", w, n4, n4)
    return -(Q[1:] - nhat * Q[0])


def _christoffel_fd(kind, a, x, h=1e-5):
    g = G.metric(kind, a, x)
    dg = torch.zeros(4, 4, 4, dtype=torch.float64)
    for d in range(3):
        dx = torch.zeros(3, dtype=torch.float64)
        dx[d] = h
        dg[:, :, d + 1] = (G.metric(kind, a, x + dx) - G.metric(kind, a, x - dx)) / (2 * h)
    low = torch.zeros(4, 4, 4, dtype=torch.float64)
    for k in range(4):
        for d in range(4):
            for s in range(4):
                low[k, d, s] = 0.5 * (dg[k, s, d] + dg[k, d, s] - dg[d, s, k])
    return torch.einsum("ek,kds->eds", torch.linalg.inv(g), low)


def _geodesic_rhs(kind, a, y):
    x, k = y[:4], y[4:]
    gam = _christoffel_fd(kind, a, x[1:])
    return torch.cat([k, -torch.einsum("mab,a,b->m", gam, k, k)])


def _tetrad_direction(kind, a, x, k):
    e = G.tetrad(kind, a, x[1:])
    kt = torch.linalg.solve(e, k)          # k^A
    return kt[1:] / kt[0]


@pytest.mark.parametrize("kind,a,p,n", [
    ("ks_sph", 0.9, (4.0, 1.0, 0.3), (0.3, -0.5, 0.81)),
    ("ks_sph", 0.9, (2.5, 2.0, 1.3), (-0.7, 0.1, 0.2)),
    ("mink_sph", 0.0, (2.0, 0.8, 0.0), (0.5, 0.5, -0.3)),
])
def test_angular_velocity_matches_geodesic(kind, a, p, n):
    """Integrate the null geodesic (RK4, Christoffels by finite differences of
    the metric) a short affine distance both ways, project its momentum onto
    the tetrad and compare d nhat / d lambda with the oracle's V."""
    x = torch.tensor((0.0,) + p, dtype=torch.float64)
    nhat = torch.tensor(n, dtype=torch.float64)
    nhat = nhat / nhat.norm()
    e = G.tetrad(kind, a, x[1:])
    k = e @ torch.cat([torch.ones(1, dtype=torch.float64), nhat])
    h, steps = 1e-3, 4

    def integrate(sign):
        y = torch.cat([x, k])
        for _ in range(steps):
            k1 = _geodesic_rhs(kind, a, y)
            k2 = _geodesic_rhs(kind, a, y + 0.5 * sign * h * k1)
            k3 = _geodesic_rhs(kind, a, y + 0.5 * sign * h * k2)
            k4 = _geodesic_rhs(kind, a, y + sign * h * k3)
            y = y + sign * h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        return _tetrad_direction(kind, a, y[:4], y[4:])

    lam = h * steps
    dn = (integrate(+1) - integrate(-1)) / (2 * lam)
    V = _angular_velocity(kind, a, x[1:], nhat)
    assert (dn - V).abs().max() < 2e-6 * max(1.0, float(V.abs().max()))


@pytest.mark.parametrize("sign", [+1, -1])
def test_kerr_circular_photon_orbit_is_fixed_direction(sign):
    """Sec. 3.3: equatorial photon orbits at r_pm = 2 + 2 cos(2/3 acos(-+a)).
    A photon on the orbit keeps its tetrad-frame direction, so V vanishes."""
    a = 0.5
    r = 2 + 2 * math.cos(2.0 / 3.0 * math.acos(-sign * a))
    x = _x((r, math.pi / 2, 0.0))
    g = G.metric("ks_sph", a, x)
    # the orbit's k ~ (1, 0, 0, Omega) must be null: solve for Omega
    A, B, Cc = float(g[3, 3]), 2 * float(g[0, 3]), float(g[0, 0])
    roots = [(-B + s * math.sqrt(B * B - 4 * A * Cc)) / (2 * A) for s in (+1, -1)]
    Om = max(roots) if sign > 0 else min(roots)
    assert abs(Om - sign / (r ** 1.5 + sign * a)) < 1e-12
    k = torch.tensor([1.0, 0.0, 0.0, Om], dtype=torch.float64)
    e = G.tetrad("ks_sph", a, x)
    kt = torch.linalg.solve(e, k)
    nhat = kt[1:] / kt[0]
    assert abs(float(nhat.norm()) - 1) < 1e-13
    V = _angular_velocity("ks_sph", a, x, nhat)
    assert V.abs().max() < 1e-13
