"""The CUDA path against closed-form solutions the paper prints for its
tests (Sec. 3), run on the GPU at the paper's sizes:

* static diffusion (Sec. 3, "Diffusion"): a Gaussian radiation pulse in a
  purely scattering static medium, alpha_s = 1e4, sigma = 0.1, intensities
  from the Minerbo closure (f <= 1/3 branch), t = 50, PLM: the L1 error of
  E against Eq. diffusion falls at least at second order in the cell count;
* advected diffusion: the same pulse in a medium moving at v = 0.02, started
  on the surface tbar = -v xbar from the fluid-frame solution and judged in
  the fluid frame at t = 50 on x in [-2, 1] (the pulse starts at x = -1);
* plane-parallel hohlraum (Sec. 3, "Hohlraums"): radiation off a wall of
  energy density 1 into vacuum, 128 cells, t = 3/4: the moment error of the
  paper's norm decreases with the number of angles.  The wall is an
  optically thick emitting slab (alpha = 1e4, source function 1/4 pi) ahead
  of x = 0, which emits the isotropic wall intensity to within O(1/(alpha dx)).
* colliding beams (Sec. 3, "Colliding Beams"): the paper's 96 x 60 grid and
  sources, beams at -+30 degrees with a 15 degree spread, t = 5/2: at the
  crossing point the intensity is bimodal (only the two beams' bins carry
  radiation), and past it each beam's flux keeps its own direction;
* beams in curvilinear coordinates (Sec. 3): the same beam (source within
  1/8 of (3/2, -1/2, 0), dI/dt = 10 within pi/8 of (1, 1, 0), t = sqrt 2) on
  64^3 cells in Cartesian coordinates and in spherical coordinates with the
  spherical tetrad (16 x 32 angles): the injected energy is conserved, and
  the energy centroid matches the semi-discrete exact value (every packet
  moves at c along its direction), closer with PLM angular reconstruction;
* beams around a spinning black hole (Sec. 3, "Beams around Black Holes"):
  a = 1/2, the paper's 62 x 5 x 256 Kerr-Schild grid, a prograde beam
  injected on the photon orbit r+ and a retrograde one on r-; at
  t = pi (r+^(3/2) + a) the prograde front has gone half an orbit and the
  retrograde one the fraction (r+^(3/2) + a) / (2 (r-^(3/2) - a)) (about a
  third).
"""
import math

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad

pytestmark = pytest.mark.gpu


def _flat_1d(level, xf):
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, level)
    d, dO, _ = rad.rad_get_angles(ctx, na)
    rad.rad_set_metric(ctx, "mink_cart", 0.0, 1, [xf, np.array([0.0, 1.0]), np.array([0.0, 1.0])],
                       (("outflow", "outflow"), ("periodic",) * 2, ("periodic",) * 2))
    return ctx, na, nap, d, dO


def _gas(M, alpha_a, alpha_s, eta):
    t = lambda a: torch.tensor(np.broadcast_to(a, (M,)).copy(), dtype=torch.float64, device="cuda").reshape(1, 1, M)
    return {"rho": t(1.0), "u": torch.zeros(1, 1, M, 3, dtype=torch.float64, device="cuda"),
            "alpha_a": t(alpha_a), "alpha_s": t(alpha_s), "eta": t(eta), "T": t(1.0)}


def _diffusion_error(N, prec, level=1, sig=0.1, a_s=1e4, t_end=50.0):
    xf = np.linspace(-1.0, 1.0, N + 1)
    ctx, na, nap, d, dO = _flat_1d(level, xf)
    try:
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(t_end / dt))
        dt = t_end / nsteps
        xc = 0.5 * (xf[1:] + xf[:-1])
        E = np.exp(-xc ** 2 / (2 * sig ** 2))
        F = xc / (3.0 * a_s * sig ** 2) * E                 # -(dE/dx) / (3 alpha_s)
        I = np.zeros((1, 1, N, nap))
        I[0, 0, :, :na] = (E[:, None] + 3.0 * d[None, :, 0] * F[:, None]) / (4 * math.pi)   # Minerbo, f <= 1/3
        tdt = torch.float64 if prec == "f64" else torch.float32
        Ig = torch.tensor(I, dtype=tdt, device="cuda")
        gas = _gas(N, 0.0, a_s, 0.0)
        o = rad.rad_opts_default(precision=rad.RAD_F64 if prec == "f64" else rad.RAD_F32,
                                 coupling=rad.RAD_COUPLE_EMISSIVITY)
        for _ in range(nsteps):
            rad.rad_step(ctx, Ig, gas, dt, o)
        torch.cuda.synchronize()
        rad.rad_check(ctx)
        Ec = (Ig[0, 0, :, :na].double().cpu().numpy() * dO[None, :]).sum(-1)
        A = (1 + 2 * t_end / (3 * a_s * sig ** 2)) ** -0.5
        Ex = A * np.exp(-A * A * xc ** 2 / (2 * sig ** 2))
        return float(np.abs(Ec - Ex).sum() * (2.0 / N))
    finally:
        rad.rad_destroy(ctx)


def test_static_diffusion_converges_to_the_papers_solution():
    errs = [_diffusion_error(N, "f64") for N in (128, 256, 512)]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5          # second order or better
    assert errs[2] < 3e-3


def test_static_diffusion_f32_matches_f64():
    e64, e32 = _diffusion_error(256, "f64"), _diffusion_error(256, "f32")
    assert abs(e32 - e64) < 0.1 * e64


def _hohlraum_error(level, N=128, nslab=16, a_wall=1e4, t_end=0.75):
    dx = 1.0 / N
    xf = np.linspace(-nslab * dx, 1.0, N + nslab + 1)
    ctx, na, nap, d, dO = _flat_1d(level, xf)
    try:
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(t_end / dt))
        dt = t_end / nsteps
        M = N + nslab
        aa = np.zeros(M)
        aa[:nslab] = a_wall
        I = np.zeros((1, 1, M, nap))
        I[0, 0, :nslab, :na] = 1.0 / (4 * math.pi)
        Ig = torch.tensor(I, dtype=torch.float64, device="cuda")
        gas = _gas(M, aa, 0.0, aa / (4 * math.pi))          # source function 1/4 pi in the wall
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        for _ in range(nsteps):
            rad.rad_step(ctx, Ig, gas, dt, o)
        torch.cuda.synchronize()
        rad.rad_check(ctx)
        Iv = Ig[0, 0, nslab:, :na].cpu().numpy()
        nx = d[:, 0]
        R = [(Iv * dO).sum(-1), (Iv * nx * dO).sum(-1), (Iv * nx * nx * dO).sum(-1)]
        s = np.clip((np.arange(N) + 0.5) * dx / t_end, 0.0, 1.0)
        exact = [0.5 * (1 - s), 0.25 * (1 - s * s), (1 - s ** 3) / 6.0]
        e = [np.abs(r - x).sum() * dx for r, x in zip(R, exact)]
        return math.sqrt(sum(v * v for v in e) / 3.0)
    finally:
        rad.rad_destroy(ctx)


def test_hohlraum_moments_converge_in_angle():
    eps = {lev: _hohlraum_error(lev) for lev in (1, 2, 4, 8)}
    assert eps[1] > eps[2] > eps[4] > eps[8]
    # at least the half order the paper expects for this discontinuous field
    assert eps[8] < eps[2] * math.sqrt(42.0 / 642.0)
    assert eps[8] < 1e-3


def _diffusion_pulse(xb, tb, sig, a_s, x0):
    A = (1 + 2 * tb / (3 * a_s * sig ** 2)) ** -0.5
    return A * np.exp(-A * A * (xb - x0) ** 2 / (2 * sig ** 2)), A


def _advected_diffusion_error(N, v=0.02, level=1, sig=0.1, a_s=1e4, t_end=50.0, x0=-1.0):
    xf = np.linspace(-2.0, 1.0, 3 * N // 2 + 1)             # N cells per two units
    ctx, na, nap, d, dO = _flat_1d(level, xf)
    try:
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(t_end / dt))
        dt = t_end / nsteps
        M = len(xf) - 1
        xc = 0.5 * (xf[1:] + xf[:-1])
        gam = 1.0 / math.sqrt(1.0 - v * v)
        ux = gam * v
        # fluid-frame state on the t = 0 surface: xbar = gam x, tbar = -gam v x
        xb, tb = gam * xc, -gam * v * xc
        Eb, A = _diffusion_pulse(xb, tb, sig, a_s, x0)
        Fb = Eb * A * A * (xb - x0) / (3.0 * a_s * sig ** 2)  # -(dEbar/dxbar) / (3 alpha_s)
        I = np.zeros((1, 1, M, nap))
        for n in range(na):
            nb0 = gam - ux * d[n, 0]                            # n^0bar = u^0 - u_x n^x
            nbx = (gam * d[n, 0] - ux) / nb0                    # fluid-frame direction cosine
            I[0, 0, :, n] = (Eb + 3.0 * nbx * Fb) / (4 * math.pi) / nb0 ** 4
        Ig = torch.tensor(I, dtype=torch.float64, device="cuda")
        gas = _gas(M, 0.0, a_s, 0.0)
        gas["u"][..., 0] = ux
        o = rad.rad_opts_default(precision=rad.RAD_F64, coupling=rad.RAD_COUPLE_EMISSIVITY)
        for _ in range(nsteps):
            rad.rad_step(ctx, Ig, gas, dt, o)
        torch.cuda.synchronize()
        rad.rad_check(ctx)
        nb0 = gam - ux * d[:, 0]
        Ebc = (Ig[0, 0, :, :na].cpu().numpy() * nb0[None, :] ** 2 * dO[None, :]).sum(-1)   # u_a u_b R^ab
        Ebx, _ = _diffusion_pulse(gam * (xc - v * t_end), gam * (t_end - v * xc), sig, a_s, x0)
        return float(np.abs(Ebc - Ebx).sum() * (xf[1] - xf[0]))
    finally:
        rad.rad_destroy(ctx)


def test_advected_diffusion_converges_to_the_papers_solution():
    errs = [_advected_diffusion_error(N) for N in (128, 256, 512)]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5
    assert errs[2] < 3e-3


def _kerr_beam_front(prograde):
    """Front angle (degrees from the source centre, along the beam) of one
    beam of the Kerr beam test at t = pi (r+^(3/2) + a), and the expected
    angle.  The grid and source are the paper's (62 x 5 x 256 cells over
    r in [1.831, 6] log-spaced, theta in [1.508, 1.634], phi in [0, 2 pi];
    source within a proper distance 7/40 of (r, pi/2, 0), beam half-opening
    5 degrees, spherical tetrad with 1hat along phi); the angles are a
    9 x 90 latitude-longitude grid (the paper's 15 x 128 exceeds the 812
    bins a step takes), whose equatorial band holds the beam directions.
    Radiation is injected into the beam bins of the source cells before
    every step (dI/dt = 70, or 60 for the retrograde beam).  The front is
    read from the midplane energy density on the orbit's ring."""
    a = 0.5
    rp = 2 + 2 * math.cos(2 / 3 * math.acos(-a))
    rm = 2 + 2 * math.cos(2 / 3 * math.acos(a))
    t_end = math.pi * (rp ** 1.5 + a)
    expect = 180.0 if prograde else 360.0 * 0.5 * (rp ** 1.5 + a) / (rm ** 1.5 - a)
    r0, rate = (rp, 70.0) if prograde else (rm, 60.0)
    nr, nth, nph = 62, 5, 256
    xf = [np.exp(np.linspace(math.log(1.831), math.log(6.0), nr + 1)), np.linspace(1.508, 1.634, nth + 1),
          np.linspace(0, 2 * math.pi, nph + 1)]
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        na, nap = rad.rad_init_angles_latlong(ctx, 9, 90)
        rad.rad_set_metric(ctx, "ks_sph", a, 3, xf,
                           (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")))
        d, dO, _ = rad.rad_get_angles(ctx, na)
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(t_end / dt))
        dt = t_end / nsteps
        rc = np.sqrt(xf[0][1:] * xf[0][:-1])
        thc, phc = 0.5 * (xf[1][1:] + xf[1][:-1]), 0.5 * (xf[2][1:] + xf[2][:-1])
        dph = np.minimum(phc, 2 * math.pi - phc) * math.sqrt(r0 * r0 + a * a + 2 * a * a / r0)
        dth, drr = (thc - math.pi / 2) * r0, (rc - r0) * math.sqrt(1 + 2 / r0)
        src = dph[:, None, None] ** 2 + dth[None, :, None] ** 2 + drr[None, None, :] ** 2 < (7 / 40) ** 2
        beam = d[:, 0] > math.cos(math.radians(5.0)) if prograde else d[:, 0] < -math.cos(math.radians(5.0))
        assert src.sum() > 10 and beam.sum() >= 1
        S = np.zeros((nph, nth, nr, nap), dtype=np.float32)
        for n in np.nonzero(beam)[0]:
            S[..., n][src] = rate * dt
        S = torch.tensor(S, device="cuda")
        I = torch.zeros_like(S)
        gas = {"rho": None, "u": None, "alpha_a": None, "alpha_s": None, "eta": None,
               "T": torch.ones((nph, nth, nr), dtype=torch.float64, device="cuda")}
        o = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_NONE)
        for _ in range(nsteps):
            I += S
            rad.rad_step(ctx, I, gas, dt, o)
        rad.rad_check(ctx)
        E = (I[..., :na].double() * torch.tensor(dO, device="cuda")).sum(-1).cpu().numpy()
    finally:
        rad.rad_destroy(ctx)
    ring = E[:, nth // 2, int(np.argmin(np.abs(rc - r0)))]
    along = np.degrees(phc) if prograde else (360.0 - np.degrees(phc)) % 360.0
    order = np.argsort(along)
    ang, e = along[order], np.log10(np.maximum(ring[order], 1e-300))
    # behind the front the beam decays exponentially along the (unstable)
    # orbit: fit that trend, and take the front where the energy first falls
    # to half of it (interpolated)
    fit = (ang > 60.0) & (ang < expect - 40.0)
    slope, icpt = np.polyfit(ang[fit], e[fit], 1)
    deficit = slope * ang + icpt - e - math.log10(2.0)
    k = np.nonzero((ang > expect - 40.0) & (deficit > 0.0))[0][0]
    x0, x1, d0, d1 = ang[k - 1], ang[k], deficit[k - 1], deficit[k]
    return x0 + (x1 - x0) * (-d0) / (d1 - d0), expect


def test_kerr_beams_travel_the_photon_orbits():
    """Sec. 3: after t = pi (r+^(3/2) + a) the prograde beam front has gone
    half an orbit and the retrograde one about a third.  Fronts within 15
    degrees of the paper's angles (the source's half-width puts them a few
    degrees ahead), and their ratio within 10 % of the paper's."""
    fp, ep = _kerr_beam_front(True)
    fr, er = _kerr_beam_front(False)
    print(f"Kerr beams: prograde front {fp:.1f} deg (paper {ep:.1f}), retrograde {fr:.1f} deg (paper {er:.1f})")
    assert abs(fp - ep) < 15.0, (fp, ep)
    assert abs(fr - er) < 15.0, (fr, er)
    assert abs((fp / fr) / (ep / er) - 1.0) < 0.10, (fp, fr, ep, er)


def test_colliding_beams_cross_without_merging():
    """Sec. 3, colliding beams: sources of radius 1/10 at x = 2/15,
    y = 1/2 +- 11/30 emit dI/dt = 5 into the directions within 7.5 degrees of
    -+30 degrees (optically thin: added every step), on the paper's 96 x 60
    grid over [0, 1.6] x [0, 1], to t = 5/2 (steady).  The angles are the
    48 in-plane directions of a 1 x 48 latitude-longitude grid, so each
    beam is two cells wide in psi, as in the paper's coarse run.  At the
    crossing point only the beams' four bins carry radiation (the
    distribution is bimodal, which a moment closure cannot represent);
    beyond it each beam's flux points along its own direction to within a
    degree, and the two beams are mirror images."""
    nx, ny = 96, 60
    xf = [np.linspace(0, 1.6, nx + 1), np.linspace(0, 1, ny + 1), np.array([0.0, 1.0])]
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        na, nap = rad.rad_init_angles_latlong(ctx, 1, 48)
        rad.rad_set_metric(ctx, "mink_cart", 0.0, 2, xf,
                           (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")))
        d, dO, _ = rad.rad_get_angles(ctx, na)
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(2.5 / dt))
        dt = 2.5 / nsteps
        xc, yc = 0.5 * (xf[0][1:] + xf[0][:-1]), 0.5 * (xf[1][1:] + xf[1][:-1])
        ang = np.arctan2(d[:, 1], d[:, 0])
        S = np.zeros((1, ny, nx, nap), dtype=np.float32)
        beams = []
        for ys, th in ((0.5 + 11 / 30, -math.pi / 6), (0.5 - 11 / 30, math.pi / 6)):
            src = (xc[None, :] - 2 / 15) ** 2 + (yc[:, None] - ys) ** 2 < 0.1 ** 2
            bins = np.abs(np.angle(np.exp(1j * (ang - th)))) < math.pi / 24 + 1e-9
            assert bins.sum() == 2 and src.sum() > 50
            for n in np.nonzero(bins)[0]:
                S[0, ..., n][src] = 5.0 * dt
            beams.append((ys, th, bins))
        S = torch.tensor(S, device="cuda")
        I = torch.zeros_like(S)
        gas = {"rho": None, "u": None, "alpha_a": None, "alpha_s": None, "eta": None,
               "T": torch.ones((1, ny, nx), dtype=torch.float64, device="cuda")}
        o = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_NONE)
        for _ in range(nsteps):
            I += S
            rad.rad_step(ctx, I, gas, dt, o)
        rad.rad_check(ctx)
        Ih = I[0, ..., :na].double().cpu().numpy()
    finally:
        rad.rad_destroy(ctx)
    E = (Ih * dO).sum(-1)
    Fx, Fy = (Ih * dO * d[:, 0]).sum(-1), (Ih * dO * d[:, 1]).sum(-1)
    cell = lambda x, y: (int(np.argmin(np.abs(yc - y))), int(np.argmin(np.abs(xc - x))))
    j, i = cell(2 / 15 + (11 / 30) / math.tan(math.pi / 6), 0.5)
    both = beams[0][2] | beams[1][2]
    assert Ih[j, i][beams[0][2]].min() > 0.3 and Ih[j, i][beams[1][2]].min() > 0.3
    assert np.abs(Ih[j, i][~both]).max() <= 1e-6 * Ih[j, i].max()
    for x in (1.2, 1.4):
        got = []
        for ys, th, _ in beams:
            j, i = cell(x, ys + (x - 2 / 15) * math.tan(th))
            assert abs(math.degrees(math.atan2(Fy[j, i], Fx[j, i]) - th)) < 1.0
            got.append(E[j, i])
        assert got[0] > 0.05 and abs(got[0] - got[1]) <= 1e-5 * got[0]


def _curvilinear_beam(kind, recon_ang=None, n=64, geodesic=None):
    """Energy, its centroid and the exact (semi-discrete) values for the
    curvilinear beam test in Cartesian ('mink_cart') or spherical
    ('mink_sph', spherical tetrad: 1hat = phi, 2hat = r, 3hat = theta)
    coordinates, on a 16 x 32 latitude-longitude grid or (geodesic = level)
    a geodesic one."""
    t_end, rate, half = math.sqrt(2.0), 10.0, math.pi / 8
    x0, beam = np.array([1.5, -0.5, 0.0]), np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    if kind == "mink_cart":
        xf = [np.linspace(1, 3, n + 1), np.linspace(-1, 1, n + 1), np.linspace(-1, 1, n + 1)]
    else:
        xf = [np.linspace(1, math.sqrt(10), n + 1), np.linspace(math.pi / 4, 3 * math.pi / 4, n + 1),
              np.linspace(-math.pi / 4, math.pi / 4, n + 1)]
    c = [0.5 * (x[1:] + x[:-1]) for x in xf]
    K, J, I_ = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    if kind == "mink_cart":
        pos = np.stack([I_, J, K], -1)
        dV = np.einsum("k,j,i->kji", np.diff(xf[2]), np.diff(xf[1]), np.diff(xf[0]))
        tet = lambda m: np.broadcast_to(np.eye(3), (m.sum(), 3, 3))
    else:
        r, th, ph = I_, J, K
        pos = np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], -1)
        dV = np.einsum("k,j,i->kji", np.diff(xf[2]), np.cos(xf[1][:-1]) - np.cos(xf[1][1:]),
                       (xf[0][1:] ** 3 - xf[0][:-1] ** 3) / 3)

        def tet(m):
            rr, tt, pp = r[m], th[m], ph[m]
            er = np.stack([np.sin(tt) * np.cos(pp), np.sin(tt) * np.sin(pp), np.cos(tt)], -1)
            et = np.stack([np.cos(tt) * np.cos(pp), np.cos(tt) * np.sin(pp), -np.sin(tt)], -1)
            ep = np.stack([-np.sin(pp), np.cos(pp), np.zeros_like(pp)], -1)
            return np.stack([ep, er, et], -2)
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        na, nap = rad.rad_init_angles(ctx, geodesic) if geodesic else rad.rad_init_angles_latlong(ctx, 16, 32)
        rad.rad_set_metric(ctx, kind, 0.0, 3, xf, (("outflow", "outflow"),) * 3)
        d, dO, _ = rad.rad_get_angles(ctx, na)
        dt = rad.rad_cfl_dt(ctx, 0.3)
        nsteps = int(math.ceil(t_end / dt))
        dt = t_end / nsteps
        src = ((pos - x0) ** 2).sum(-1) < (1 / 8) ** 2
        ncart = np.einsum("cAx,nA->cnx", tet(src), d)          # bin directions in Cartesian, source cells
        inb = (ncart @ beam) > math.cos(half)
        w = inb * dO * dV[src][:, None]
        E_exact = rate * t_end * w.sum()
        cen_exact = (w[..., None] * (pos[src][:, None, :] + 0.5 * t_end * ncart)).sum((0, 1)) / w.sum()
        S = np.zeros((n, n, n, nap), dtype=np.float32)
        S[src] = np.concatenate([np.where(inb, rate * dt, 0.0), np.zeros((src.sum(), nap - na))], -1)
        S = torch.tensor(S, device="cuda")
        I = torch.zeros_like(S)
        gas = {"rho": None, "u": None, "alpha_a": None, "alpha_s": None, "eta": None,
               "T": torch.ones((n, n, n), dtype=torch.float64, device="cuda")}
        o = rad.rad_opts_default(precision=rad.RAD_F32, coupling=rad.RAD_COUPLE_NONE,
                                 recon_ang=recon_ang if recon_ang is not None else rad.RAD_RECON_DC)
        for _ in range(nsteps):
            I += S
            rad.rad_step(ctx, I, gas, dt, o)
        rad.rad_check(ctx)
        E = (I[..., :na].double() * torch.tensor(dO, device="cuda")).sum(-1).cpu().numpy() * dV
    finally:
        rad.rad_destroy(ctx)
    cen = (E[..., None] * pos).sum((0, 1, 2)) / E.sum()
    return E.sum(), E_exact, float(np.linalg.norm(cen - cen_exact))


def test_mapr_beam_is_less_diffusive_than_donor_cell():
    """Sec. 3: the paper shows minimum-angle plane reconstruction reducing
    the angular diffusion of a beam whose angular fluxes come from the
    coordinates (its snake-coordinate test); here the curvilinear beam in
    spherical coordinates on a level-7 geodesic grid (492 bins): energy
    conserved to 1e-5 either way, and the centroid closer to the exact value
    with MAPR than with donor-cell angular fluxes."""
    Ed, Ede, dd = _curvilinear_beam("mink_sph", rad.RAD_RECON_DC, geodesic=7)
    Em, Eme, dm = _curvilinear_beam("mink_sph", rad.RAD_RECON_MAPR, geodesic=7)
    print(f"geodesic beam: centroid offsets {dd:.4f} (DC) {dm:.4f} (MAPR)")
    for E, Ee in ((Ed, Ede), (Em, Eme)):
        assert abs(E / Ee - 1.0) < 1e-5
    assert dm < dd


def test_curvilinear_beam_is_the_same_in_cartesian_and_spherical_coordinates():
    """Sec. 3, beams in curvilinear coordinates: energy conserved to 1e-5 in
    both coordinate systems (the beam stays inside the domain), centroid
    within 0.01 (Cartesian) and 0.03 (spherical, where the angular fluxes
    add the anisotropic numerical diffusion the paper notes) of the exact
    value, and closer with PLM than with DC angular reconstruction."""
    Ec, Ece, dc = _curvilinear_beam("mink_cart")
    Es, Ese, ds = _curvilinear_beam("mink_sph")
    Ep, Epe, dp = _curvilinear_beam("mink_sph", rad.RAD_RECON_PLM)
    print(f"curvilinear beam: centroid offsets Cartesian {dc:.4f}, spherical {ds:.4f} (DC) {dp:.4f} (PLM)")
    for E, Ee in ((Ec, Ece), (Es, Ese), (Ep, Epe)):
        assert abs(E / Ee - 1.0) < 1e-5
    assert dc < 0.01 and ds < 0.03 and dp < ds
