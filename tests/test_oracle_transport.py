"""Pins of the oracle's transport (Secs. 2.2-2.4, Eq. flux_space, Eq.
flux_angle, Eq. radiation_integral) and of its RK2 step: exact invariants,
exact beam speed, brute-force hand expansion and the hohlraum closed form
(Sec. 3.4)."""
import math

import numpy as np
import pytest
import torch

from oracle import step as S
from oracle import transport as TR
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup

F64 = torch.float64


def cart_setup(n, level, ndim, L=1.0, bc="periodic"):
    ang = GeodesicGrid(level)
    xf = [np.linspace(0, L, n[d] + 1) if d < ndim else np.array([0.0, 1.0]) for d in range(3)]
    grid = Grid("mink_cart", 0.0, xf, ((bc, bc),) * 3, ndim)
    return Setup(grid, ang)


@pytest.fixture(scope="module")
def ks_setup():
    ang = GeodesicGrid(2)
    xf = [np.exp(np.linspace(math.log(1.6), math.log(8.0), 7)), np.linspace(0, math.pi, 7),
          np.linspace(0, 2 * math.pi, 5)]
    grid = Grid("ks_sph", 0.9, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), 3)
    return Setup(grid, ang)


@pytest.mark.parametrize("recon", ["dc", "plm"])
def test_uniform_field_is_stationary_in_flat_space(recon):
    st = cart_setup((6, 5, 4), 2, 3)
    I = torch.full(st.grid.shape + (st.ang.n_ang,), 0.37, dtype=F64)
    L = S.operator_L(I, st, S.Opts(recon=recon))
    assert L.abs().max() < 1e-14


@pytest.mark.parametrize("recon", ["dc", "plm"])
def test_conservation_periodic(recon):
    """sum dV U is conserved to roundoff by the finite-volume form (Sec. 2.2)."""
    st = cart_setup((6, 5, 4), 2, 3)
    rng = np.random.default_rng(7)
    I = torch.tensor(rng.uniform(0.5, 1.5, st.grid.shape + (st.ang.n_ang,)))
    L = S.operator_L(I, st, S.Opts(recon=recon))
    assert abs(float((L * st.dV[..., None]).sum())) < 1e-14 * float((I * st.dV[..., None]).sum())


def test_angular_fluxes_conserve_per_cell(ks_setup):
    rng = np.random.default_rng(3)
    I = torch.tensor(rng.uniform(0.5, 1.5, ks_setup.grid.shape + (ks_setup.ang.n_ang,)))
    divA = TR.angular_divergence(I, ks_setup)
    tot = (divA * ks_setup.ang.dOmega).sum(-1)
    assert tot.abs().max() < 1e-13 * float(divA.abs().max())
    assert divA.abs().max() > 1e-3           # the fluxes are not trivially zero


def test_no_angular_flux_in_cartesian_minkowski():
    st = cart_setup((4, 4, 1), 2, 2)
    I = torch.rand(st.grid.shape + (st.ang.n_ang,), dtype=F64)
    assert TR.angular_divergence(I, st).abs().max() == 0.0


def test_beam_centroid_moves_at_light_speed():
    """DC upwind is conservative with a consistent linear flux, so the first
    moment of a beam in one bin moves exactly at n^x / n^0 = nhat^x per unit
    time (the RK2 integration of a linear first moment is exact)."""
    st = cart_setup((64, 1, 1), 2, 1, L=1.0)
    n = int(torch.argmax(st.ang.dir[:, 0]))
    I = torch.zeros(st.grid.shape + (st.ang.n_ang,), dtype=F64)
    I[0, 0, 10:20, n] = 1.0
    x = torch.tensor(st.grid.xc[0])
    opts = S.Opts(recon="dc", couple=False)
    dt = 0.4 / 64
    gas = None
    t = 0.0
    m0 = float((I[0, 0, :, n] * x).sum() / I[0, 0, :, n].sum())
    for _ in range(20):
        I, _, _, _ = S.rk2_step(I, torch.zeros(st.grid.shape, dtype=F64), gas, dt, st, opts)
        t += dt
    m1 = float((I[0, 0, :, n] * x).sum() / I[0, 0, :, n].sum())
    assert abs((m1 - m0) - float(st.ang.dir[n, 0]) * t) < 1e-13
    # other bins stay empty
    others = torch.ones(st.ang.n_ang, dtype=torch.bool)
    others[n] = False
    assert I[..., others].abs().max() == 0.0


def test_brute_force_two_cells_hand_expanded():
    """2x1x1 periodic cells, level 1, DC: each face flux is -nhat^x I_upwind and
    L_i = -(F_{i+1/2} - F_{i-1/2}) / dx, expanded by hand per bin."""
    st = cart_setup((2, 1, 1), 1, 1, L=2.0)
    rng = np.random.default_rng(1)
    I = torch.tensor(rng.uniform(0.1, 1.0, (1, 1, 2, 12)))
    L = S.operator_L(I, st, S.Opts(recon="dc"))
    dx = 1.0
    for n in range(12):
        c = float(st.ang.dir[n, 0])
        I0, I1 = float(I[0, 0, 0, n]), float(I[0, 0, 1, n])
        # U = n^0 n_0 I = -I, flux of U through x faces = n^x n_0 I_up = -c I_up
        up_left_face = I1 if c > 0 else I0     # face between cell 1 (periodic image) and cell 0
        up_mid_face = I0 if c > 0 else I1
        F_lo, F_mid = -c * up_left_face, -c * up_mid_face
        assert abs(float(L[0, 0, 0, n]) + (F_mid - F_lo) / dx) < 1e-15
        assert abs(float(L[0, 0, 1, n]) + (F_lo - F_mid) / dx) < 1e-15


def test_plm_reproduces_linear_profile_slopes():
    """van Leer's harmonic mean of equal one-sided differences is the difference itself."""
    dl = torch.tensor([0.3, -0.2, 0.5, 0.0], dtype=F64)
    dr = torch.tensor([0.3, -0.2, -0.1, 0.4], dtype=F64)
    s = TR.van_leer(dl, dr)
    assert torch.allclose(s, torch.tensor([0.3, -0.2, 0.0, 0.0], dtype=F64), atol=0, rtol=1e-15)


def _hohlraum_error(level, ncell=64, t_end=0.5, ang=None):
    """1D hohlraum (Sec. 3.4): an isotropic wall of energy density 1 at x = 0."""
    ang = GeodesicGrid(level) if ang is None else ang
    xf = [np.linspace(0, 1, ncell + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    grid = Grid("mink_cart", 0.0, xf, (("outflow", "outflow"),) * 3, 1)
    st = Setup(grid, ang)
    I = torch.zeros(grid.shape + (ang.n_ang,), dtype=F64)
    wall = 1.0 / (4 * math.pi)
    dt = 0.4 / ncell
    nsteps = int(round(t_end / dt))

    def L(I):
        Ie = TR.fill_ghosts(I, grid, ang.perm_pi2)
        Ie[:, :, :TR.NG, :] = wall              # the wall held fixed
        return -TR.spatial_divergence(Ie, st, "plm")

    f = st.f
    for _ in range(nsteps):
        U0 = f * I
        I1 = (U0 + dt * L(I)) / f
        I = (0.5 * U0 + 0.5 * (f * I1 + dt * L(I1))) / f
    t = nsteps * dt
    x = torch.tensor(grid.xc[0])
    xi = torch.clamp(x / t, max=1.0)
    n4 = torch.cat([torch.ones(ang.n_ang, 1, dtype=F64), ang.dir], 1)
    R = torch.einsum("kjin,nA,nB,n->iAB", I, n4, n4, ang.dOmega)
    exact = [0.5 * (1 - xi), 0.25 * (1 - xi ** 2), (1 - xi ** 3) / 6.0]
    dxx = 1.0 / ncell
    eps = [float((R[:, 0, 0] - exact[0]).abs().sum() * dxx),
           float((R[:, 0, 1] - exact[1]).abs().sum() * dxx),
           float((R[:, 1, 1] - exact[2]).abs().sum() * dxx)]
    return math.sqrt(sum(e * e for e in eps) / 3.0)


def test_hohlraum_converges_in_angle():
    """Sec. 3.4: R^tt = (1 - x/t)/2, R^tx = (1 - x^2/t^2)/4, R^xx = (1 - x^3/t^3)/6;
    the error falls with the number of angles (about N_ang^(-1/2))."""
    e = [_hohlraum_error(N) for N in (1, 2, 4)]
    assert e[0] > e[1] > e[2]
    assert e[2] < 0.03


def test_hohlraum_converges_in_angle_on_latlong_grids():
    """The same closed forms with latitude-longitude grids (Sec. 2.6) of
    3 x 6, 6 x 12 and 12 x 24 angles."""
    from oracle.angles import LatLongGrid
    e = [_hohlraum_error(0, ang=LatLongGrid(nz, 2 * nz)) for nz in (3, 6, 12)]
    assert e[0] > e[1] > e[2]
    assert e[2] < 0.03


@pytest.mark.parametrize("recon_ang", ["dc", "plm"])
def test_latlong_angular_fluxes_conserve_per_cell(recon_ang):
    """Kerr-Schild with a latitude-longitude grid: the angular fluxes only
    move intensity between bins of a cell (DC and PLM along the grid lines)."""
    from oracle.angles import LatLongGrid
    ang = LatLongGrid(4, 8)
    xf = [np.exp(np.linspace(math.log(1.6), math.log(8.0), 7)), np.linspace(0, math.pi, 7),
          np.linspace(0, 2 * math.pi, 5)]
    grid = Grid("ks_sph", 0.9, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), 3)
    st = Setup(grid, ang)
    rng = np.random.default_rng(4)
    I = torch.tensor(rng.uniform(0.5, 1.5, grid.shape + (ang.n_ang,)))
    divA = TR.angular_divergence(I, st, recon_ang)
    tot = (divA * ang.dOmega).sum(-1)
    assert tot.abs().max() < 1e-13 * float(divA.abs().max())
    assert divA.abs().max() > 1e-3


# ---------------------------------------------- optical-depth flux weighting
def _tau_case(n=(6, 5, 4), level=2, seed=21, umax=0.4):
    st = cart_setup(n, level, 3)
    rng = np.random.default_rng(seed)
    sh = st.grid.shape
    v = rng.uniform(-1, 1, sh + (3,))
    v *= umax / np.sqrt((v * v).sum(-1)).max()
    gas = {"u": torch.tensor(v / np.sqrt(1 - (v * v).sum(-1))[..., None]),
           "alpha_a": torch.tensor(10.0 ** rng.uniform(-1, 2, sh)),
           "alpha_s": torch.tensor(10.0 ** rng.uniform(-1, 2, sh))}
    I = torch.tensor(rng.uniform(0.5, 1.5, sh + (st.ang.n_ang,)))
    return st, gas, I


def _L_tau(st, gas, I, C, dt=0.01, recon="plm"):
    tau = TR.tau_weights(st, gas, dt, C)
    return S.operator_L(I, st, S.Opts(recon=recon), tau)


def test_tau_weighting_with_zero_constant_is_free_streaming():
    """Sec. 2.4: a proportionality constant of 0 reduces to the free-streaming flux."""
    st, gas, I = _tau_case()
    assert torch.equal(_L_tau(st, gas, I, 0.0), S.operator_L(I, st, S.Opts()))


@pytest.mark.parametrize("uniform", [False, True])
def test_tau_weighting_is_inactive_for_static_or_uniform_gas(uniform):
    """With the same velocity on both sides of every face, n^0bar_L = n^0bar_R,
    so g_L = g_R = g and both factors are exactly 1, whatever the optical depth."""
    st, gas, I = _tau_case()
    u = gas["u"]
    gas["u"] = u[:1, :1, :1].expand_as(u).clone() if uniform else torch.zeros_like(u)
    L0 = S.operator_L(I, st, S.Opts())
    assert (_L_tau(st, gas, I, 5.0) - L0).abs().max() <= 1e-14 * L0.abs().max()


def test_tau_weighting_conserves_with_periodic_boundaries():
    """Each face carries one flux (the weights are per face), so sum dV U is
    still conserved to roundoff, and the weighting does change the fluxes."""
    st, gas, I = _tau_case()
    L = _L_tau(st, gas, I, 3.0)
    assert abs(float((L * st.dV[..., None]).sum())) < 1e-13 * float((I * st.dV[..., None]).sum())
    assert (L - S.operator_L(I, st, S.Opts())).abs().max() > 1e-3 * L.abs().max()


def test_tau_weighting_is_quadratic_in_small_optical_depth():
    """f = -expm1(-tau^2) = tau^2 (1 + O(tau^2)): for small optical depth the
    departure of every weight from 1 is quadratic in C (ratio 4 when C
    doubles), and it is not identically zero for a moving gas."""
    st, gas, I = _tau_case()
    w1 = TR.tau_weights(st, gas, 1e-2, 1e-3)     # tau <= 2e-3: O(tau^2) terms below 1e-5
    w2 = TR.tau_weights(st, gas, 1e-2, 2e-3)
    for d in range(3):
        for side in (0, 1):
            a, b = w1[d][side] - 1.0, w2[d][side] - 1.0
            big = a.abs() > 1e-2 * a.abs().max()
            assert float(a.abs().max()) > 1e-10
            assert float((b[big] / a[big] - 4.0).abs().max()) < 1e-4


# ------------------------------------------------ PPM (Colella & Woodward 1984)
def _ppm_line(vals):
    line = torch.tensor(vals, dtype=F64)[:, None]          # [cells, 1]
    return TR.ppm_edges(line, 0)


def test_ppm_interfaces_are_exact_for_linear_and_quadratic_data():
    """Cell averages of a linear or (monotone) quadratic profile: the
    interface values equal the profile's point values there (the method's
    fourth-order interface formula is exact for cubics), and no constraint
    fires inside a monotone parabola."""
    x = np.arange(12, dtype=float)                          # cell j spans [j, j+1]
    lin = 0.5 + 2.0 * (x + 0.5)
    aL, aR = _ppm_line(lin)
    faces = np.arange(2, 10, dtype=float)                   # cells 2..9: left faces at x = 2..9
    assert np.allclose(aL[:, 0].numpy(), 0.5 + 2.0 * faces, rtol=0, atol=1e-13)
    assert np.allclose(aR[:, 0].numpy(), 0.5 + 2.0 * (faces + 1), rtol=0, atol=1e-13)
    f = lambda z: 3.0 + 0.3 * z + 0.05 * z * z              # monotone on z >= 0
    avg = np.array([(lambda a, b: (0.15 * (b * b - a * a) + 0.05 * (b ** 3 - a ** 3) / 3 + 3.0) / 1.0)(j, j + 1.0)
                    for j in x])
    aL, aR = _ppm_line(avg)
    assert np.allclose(aL[:, 0].numpy(), f(faces), rtol=0, atol=1e-12)
    assert np.allclose(aR[:, 0].numpy(), f(faces + 1), rtol=0, atol=1e-12)


def test_ppm_creates_no_new_extrema():
    """Edge values of every cell stay within the range of the cell and its
    neighbours (monotonicity), for a step, a spike and random data; at a
    local extremum the parabola is flattened to the cell value."""
    rng = np.random.default_rng(13)
    for vals in (np.r_[np.zeros(6), np.ones(6)], np.r_[np.zeros(5), [1.0], np.zeros(6)], rng.uniform(0, 1, 40)):
        aL, aR = _ppm_line(vals)
        a = vals[2:-2]
        lo = np.minimum(np.minimum(vals[1:-3], vals[2:-2]), vals[3:-1])
        hi = np.maximum(np.maximum(vals[1:-3], vals[2:-2]), vals[3:-1])
        for e in (aL[:, 0].numpy(), aR[:, 0].numpy()):
            assert (e >= lo - 1e-14).all() and (e <= hi + 1e-14).all()
        ext = ((vals[3:-1] - a) * (a - vals[1:-3])) <= 0
        assert np.allclose(aL[:, 0].numpy()[ext], a[ext]) and np.allclose(aR[:, 0].numpy()[ext], a[ext])


def test_ppm_step_is_conservative_and_keeps_uniform_fields():
    st = cart_setup((6, 5, 4), 2, 3)
    I = torch.full(st.grid.shape + (st.ang.n_ang,), 0.37, dtype=F64)
    assert S.operator_L(I, st, S.Opts(recon="ppm")).abs().max() < 1e-14
    rng = np.random.default_rng(7)
    I = torch.tensor(rng.uniform(0.5, 1.5, st.grid.shape + (st.ang.n_ang,)))
    L = S.operator_L(I, st, S.Opts(recon="ppm"))
    assert abs(float((L * st.dV[..., None]).sum())) < 1e-14 * float((I * st.dV[..., None]).sum())


def test_ppm_beam_is_more_accurate_than_plm():
    """A smooth 1D pulse advected along +x by one bin: after a fixed time the
    PPM solution is closer to the exact translate than PLM's, and both
    converge under refinement."""
    errs = {}
    for recon in ("plm", "ppm"):
        for n in (32, 64):
            ang = GeodesicGrid(1)
            xf = [np.linspace(0, 1, n + 1), np.array([0.0, 1.0]), np.array([0.0, 1.0])]
            st = Setup(Grid("mink_cart", 0.0, xf, (("periodic", "periodic"),) * 3, 1), ang)
            nx = st.ang.dir[:, 0].numpy()
            b = int(np.argmax(nx))                           # the bin closest to +x
            xc = 0.5 * (xf[0][1:] + xf[0][:-1])
            prof = lambda x: np.exp(-((x - 0.5) / 0.1) ** 2)
            I = torch.zeros(st.grid.shape + (st.ang.n_ang,), dtype=F64)
            I[0, 0, :, b] = torch.tensor(prof(xc))
            dt = 0.3 / n
            t_end = 0.25 / nx[b]                              # the pulse moves 0.25 in x
            steps = int(round(t_end / dt))
            for _ in range(steps):
                I, _, _, _ = S.rk2_step(I, torch.ones(st.grid.shape, dtype=F64), _no_gas(st.grid.shape), dt, st,
                                        S.Opts(recon=recon, couple=False))
            shift = nx[b] * dt * steps
            exact = prof(((xc - shift) % 1.0))
            errs[(recon, n)] = float(np.abs(I[0, 0, :, b].numpy() - exact).mean())
    assert errs[("ppm", 64)] < errs[("plm", 64)]
    assert errs[("ppm", 64)] < 0.5 * errs[("ppm", 32)]


def _no_gas(sh):
    z = torch.zeros(sh, dtype=F64)
    return {"rho": z + 1.0, "u": torch.zeros(sh + (3,), dtype=F64), "alpha_a": z, "alpha_s": z, "eta": None}
