"""Pins of the oracle's minimum-angle plane reconstruction (MAPR) of angular
face values on geodesic grids (Sec. 2.6 names the method; the reading of it
is stated in oracle.transport.mapr_face_values): exact values for data that
are linear in a cell's gnomonic tangent coordinates, the chosen plane
against a brute-force search over the candidate planes, constant data, and
per-cell conservation of the angular fluxes."""
import math

import numpy as np
import pytest
import torch

from oracle import step as S
from oracle import transport as TR
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup


def _tangent(n):
    # an orthonormal pair normal to n, built here independently of the oracle's
    t1 = np.cross(n, [0.0, 0.0, 1.0]) if abs(n[2]) < 0.9 else np.cross(n, [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1)
    return t1, np.cross(n, t1)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_linear_data_are_reproduced_exactly(level):
    """I = alpha + beta . x on cell c and its neighbours (x: gnomonic
    coordinates at c) makes every candidate plane exact, so c's value at each
    side is alpha + beta . x_side, whatever the basis of the tangent plane."""
    ang = GeodesicGrid(level)
    dirs, mids = ang.dir.numpy(), ang.edge_mid.numpy()
    rng = np.random.default_rng(level)
    for c in rng.choice(ang.n_ang, size=min(8, ang.n_ang), replace=False):
        n = dirs[c]
        t1, t2 = _tangent(n)
        gn = lambda v: np.array([v @ t1, v @ t2]) / (v @ n)
        alpha, beta = rng.uniform(1, 2), rng.normal(size=2)
        I = rng.uniform(0.5, 1.5, ang.n_ang)
        for m in [c] + list(ang.nbr[c]):
            I[m] = alpha + beta @ gn(dirs[m])
        Fp, Fq = TR.mapr_face_values(torch.tensor(I), ang)
        for e, (p, q) in enumerate(ang.edges.tolist()):
            if c in (p, q):
                got = float((Fp if p == c else Fq)[e])
                assert abs(got - (alpha + beta @ gn(mids[e]))) < 1e-12


def test_chosen_plane_has_the_smallest_gradient():
    """Brute force: all planes through c and two cyclically adjacent
    neighbours (numpy least squares), the flattest one evaluated at c's
    sides, against the oracle's values, on random data."""
    ang = GeodesicGrid(2)
    dirs, mids = ang.dir.numpy(), ang.edge_mid.numpy()
    rng = np.random.default_rng(11)
    I = rng.uniform(0.5, 1.5, ang.n_ang)
    Fp, Fq = TR.mapr_face_values(torch.tensor(I), ang)
    for c in range(ang.n_ang):
        n = dirs[c]
        t1, t2 = _tangent(n)
        gn = lambda v: np.array([v @ t1, v @ t2]) / (v @ n)
        nb = sorted(ang.nbr[c], key=lambda m: math.atan2(gn(dirs[m])[1], gn(dirs[m])[0]))
        best = None
        for a in range(len(nb)):
            b = nb[(a + 1) % len(nb)]
            A = np.array([gn(dirs[nb[a]]), gn(dirs[b])])
            g = np.linalg.lstsq(A, np.array([I[nb[a]] - I[c], I[b] - I[c]]), rcond=None)[0]
            if best is None or g @ g < best @ best:
                best = g
        for e, (p, q) in enumerate(ang.edges.tolist()):
            if c in (p, q):
                got = float((Fp if p == c else Fq)[e])
                assert abs(got - (I[c] + best @ gn(mids[e]))) < 1e-12


def test_constant_data_give_the_cell_value():
    ang = GeodesicGrid(2)
    Fp, Fq = TR.mapr_face_values(torch.full((ang.n_ang,), 0.7, dtype=torch.float64), ang)
    assert float((Fp - 0.7).abs().max()) < 1e-15 and float((Fq - 0.7).abs().max()) < 1e-15


def test_mapr_angular_fluxes_conserve_per_cell():
    """The sum over bins of dOmega divA vanishes in every cell (each side's
    flux leaves one bin and enters the other), on Kerr-Schild with MAPR."""
    ang = GeodesicGrid(2)
    xf = [np.exp(np.linspace(math.log(1.6), math.log(8.0), 5)), np.linspace(0, math.pi, 5),
          np.linspace(0, 2 * math.pi, 5)]
    st = Setup(Grid("ks_sph", 0.9, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), 3), ang)
    rng = np.random.default_rng(3)
    I = torch.tensor(rng.uniform(0.5, 1.5, st.grid.shape + (ang.n_ang,)))
    div = TR.angular_divergence(I, st, "mapr")
    dc = TR.angular_divergence(I, st, "dc")
    tot = (div * ang.dOmega).sum(-1)
    assert tot.abs().max() < 1e-13 * float(div.abs().max())
    assert float((div - dc).abs().max()) > 1e-3 * float(dc.abs().max())   # the reconstruction acts
    # constant data: MAPR fluxes are the donor-cell ones
    I1 = torch.full_like(I, 0.4)
    assert float((TR.angular_divergence(I1, st, "mapr") - TR.angular_divergence(I1, st, "dc")).abs().max()) < 1e-15


def test_mapr_is_refused_on_latlong_grids():
    from oracle.angles import LatLongGrid
    ang = LatLongGrid(3, 6)
    with pytest.raises(ValueError):
        TR.angular_face_values(torch.ones(ang.n_ang, dtype=torch.float64), ang, "mapr")


def test_mapr_gradient_matches_central_differences():
    """Away from ties the chosen plane is locally fixed, so the step is
    differentiable: reverse-mode AD of the oracle against central differences
    of its forward (2D Kerr-Schild, level-2 geodesic grid, two steps) in
    alpha_a and in intensities."""
    import workloads as W
    from oracle import adjoint as A
    from oracle import cfl as CF
    w = W.make("adjoint2d", n=(6, 4, 1), level=2)
    ang = GeodesicGrid(2)
    st = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), ang)
    gas = {k: (torch.tensor(w[k]) if w[k] is not None else None)
           for k in ("rho", "u", "alpha_a", "alpha_s", "eta")}
    dt = CF.cfl_dt(st, 0.3)
    opts = S.Opts(mode="emissivity", recon_ang="mapr")
    I0, T0 = torch.tensor(w["I0"]), torch.tensor(w["T"])
    nsteps = 2
    _, grads = A.gradient(I0, T0, gas, dt, st, opts, nsteps)
    I0r = I0.clone().requires_grad_(True)
    I, T = I0r, T0
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

    checks = [("alpha_a", grads[0], gas["alpha_a"], (0, 1, 5)), ("alpha_a", grads[0], gas["alpha_a"], (0, 3, 4))]
    for idx in [(0, 1, 5, 3), (0, 2, 5, 17), (0, 3, 4, 30)]:
        checks.append(("I", gI, I0, idx))
    for field, grad, base, idx in checks:
        gmax = float(grad.abs().max())
        h = 1e-6 * max(abs(float(base[idx])), 1e-3 * float(base.abs().max()))
        fd = (loss_with(field, idx, h) - loss_with(field, idx, -h)) / (2 * h)
        ad = float(grad[idx])
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 2e-2 * gmax), (field, idx, fd, ad)

