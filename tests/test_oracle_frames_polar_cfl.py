"""Pins of three oracle functions against facts fixed outside the oracle:

* the coordinate-frame moments R^{mu nu} = e^mu_A e^nu_B R^{AB} (Sec. 2.5,
  the definition of R), against the closed forms of flat spherical
  coordinates with the spherical tetrad (Sec. 2.1's tetrad: 3hat along
  theta, 1hat along phi, 2hat along r) and, in Kerr-Schild, against the
  metric trace and the lowered moments written from n^mu and n_mu;
* the polar ghost fill (the boundary task of Sec. 2, reading R18), cell by
  cell against a field defined by physical position and physical direction:
  a ghost cell at theta < 0 or theta > pi is the point reached by continuing
  the coordinates through the axis, and its bins are directions expressed in
  the tetrad continued smoothly through the axis, so its value must be the
  field's value there;
* the angular part of the time-step bound (reading R10), against the rate
  of change of a straight ray's direction in the rotating spherical frame,
  derived by hand below.
"""
import math

import numpy as np
import torch

from oracle import cfl as CF
from oracle import moments as M
from oracle import transport as TR
from oracle.angles import GeodesicGrid, LatLongGrid
from oracle.transport import Grid, Setup

F64 = torch.float64


def _sph_grid(n1, n2, n3, r0=2.0, r1=5.0, kind="mink_sph", a=0.0, ndim=3):
    xf = [np.linspace(r0, r1, n1 + 1), np.linspace(0.0, math.pi, n2 + 1), np.linspace(0.0, 2 * math.pi, n3 + 1)]
    return Grid(kind, a, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), ndim)


# ------------------------------------------------------------------ moments
def test_coordinate_moments_flat_spherical_closed_form():
    """With the spherical tetrad in flat space e^r_2hat = 1, e^theta_3hat = 1/r,
    e^phi_1hat = 1/(r sin theta), e^t_0hat = 1, so
    R^{tt} = R^{00hat}, R^{tr} = R^{02hat}, R^{rr} = R^{22hat},
    R^{theta theta} = R^{33hat}/r^2, R^{phi phi} = R^{11hat}/(r^2 sin^2 theta),
    R^{r theta} = R^{23hat}/r, R^{r phi} = R^{21hat}/(r sin theta),
    R^{theta phi} = R^{31hat}/(r^2 sin theta), R^{t theta} = R^{03hat}/r,
    R^{t phi} = R^{01hat}/(r sin theta)."""
    grid = _sph_grid(3, 4, 2)
    ang = GeodesicGrid(3)
    st = Setup(grid, ang)
    rng = np.random.default_rng(11)
    I = torch.tensor(rng.uniform(0.1, 1.0, grid.shape + (ang.n_ang,)))
    Rt = M.tetrad_moments(I, ang)                              # [..., A, B]
    Rc = M.moments(I, ang, "coord", e=st.e)                    # 10 components, coordinate order
    X = grid.centres()
    r, th = X[..., 0], X[..., 1]
    s = torch.sin(th)
    T = lambda A, B: Rt[..., A, B]
    ref = {  # (mu, nu) in (t, r, theta, phi) = (0, 1, 2, 3)
        (0, 0): T(0, 0), (0, 1): T(0, 2), (0, 2): T(0, 3) / r, (0, 3): T(0, 1) / (r * s),
        (1, 1): T(2, 2), (1, 2): T(2, 3) / r, (1, 3): T(2, 1) / (r * s),
        (2, 2): T(3, 3) / r ** 2, (2, 3): T(3, 1) / (r * r * s), (3, 3): T(1, 1) / (r * s) ** 2,
    }
    for c, pair in enumerate(M.PAIRS):
        err = (Rc[..., c] - ref[pair]).abs().max() / ref[pair].abs().max().clamp_min(1e-300)
        assert err < 1e-13, (pair, float(err))


def test_coordinate_moments_kerr_schild_trace_and_lowered_row():
    """In Kerr-Schild (a = 0.9): g_{mu nu} R^{mu nu} = eta_{AB} R^{AB} = 0 for
    null directions, and R^0_mu = g_{mu nu} R^{0 nu} equals the definition
    sum_n I_n n^0 n_mu dOmega_n written with the oracle's n^mu and n_mu."""
    grid = _sph_grid(3, 4, 2, r0=1.6, r1=8.0, kind="ks_sph", a=0.9)
    ang = GeodesicGrid(2)
    st = Setup(grid, ang)
    rng = np.random.default_rng(12)
    I = torch.tensor(rng.uniform(0.1, 1.0, grid.shape + (ang.n_ang,)))
    R10 = M.moments(I, ang, "coord", e=st.e)
    R = torch.zeros(grid.shape + (4, 4), dtype=F64)
    for c, (a, b) in enumerate(M.PAIRS):
        R[..., a, b] = R10[..., c]
        R[..., b, a] = R10[..., c]
    trace = torch.einsum("...mn,...mn->...", st.g, R)
    assert trace.abs().max() < 1e-12 * R[..., 0, 0].abs().max()
    lowered = torch.einsum("...mv,...v->...m", st.g, R[..., 0, :])
    direct = torch.einsum("...n,...n,...nm,n->...m", I, st.nup[..., 0], st.nlow, ang.dOmega)
    assert (lowered - direct).abs().max() < 1e-12 * direct.abs().max()
    # and the energy density seen by the normal observer is the tetrad R^{00}
    Rt = M.tetrad_moments(I, ang)
    e0 = st.e[..., :, 0]                                   # e_0hat^mu
    gl = torch.einsum("...mv,...v->...m", st.g, e0)        # its lowered form
    E = torch.einsum("...m,...n,...mn->...", gl, gl, R)
    assert (E - Rt[..., 0, 0]).abs().max() < 1e-12 * Rt[..., 0, 0].abs().max()


# --------------------------------------------------------------- polar fill
def _frame(th, ph):
    """Flat spherical orthonormal frame continued smoothly through the axis:
    e_r, e_theta, e_phi as Cartesian vectors (valid for any theta)."""
    er = torch.stack([torch.sin(th) * torch.cos(ph), torch.sin(th) * torch.sin(ph), torch.cos(th)], -1)
    et = torch.stack([torch.cos(th) * torch.cos(ph), torch.cos(th) * torch.sin(ph), -torch.sin(th)], -1)
    ep = torch.stack([-torch.sin(ph), torch.cos(ph), torch.zeros_like(ph)], -1)
    return er, et, ep


def _field(pos, nvec):
    """An arbitrary smooth field of position and direction with no symmetry."""
    x, y, z = pos[..., 0:1], pos[..., 1:2], pos[..., 2:3]
    nx, ny, nz = nvec[..., 0], nvec[..., 1], nvec[..., 2]
    return (1.5 + 0.3 * torch.sin(1.3 * x + 0.4) * torch.cos(0.7 * y - 0.2) + 0.2 * z
            + 0.25 * nx - 0.15 * ny + 0.35 * nz + 0.1 * nx * nz + 0.05 * (x + 2 * y) * ny)


def _sample(r, th, ph, dirs):
    """Field at cell centre (r, th, ph) for every bin: bin components are
    (1hat, 2hat, 3hat) = (phi, r, theta) of the spherical tetrad."""
    er, et, ep = _frame(th, ph)
    pos = r[..., None] * er
    nvec = (dirs[:, 0, None] * ep[..., None, :] + dirs[:, 1, None] * er[..., None, :]
            + dirs[:, 2, None] * et[..., None, :])
    return _field(pos, nvec)


def _check_polar_ghosts(ang, n1=3, n2=6, n3=8):
    grid = _sph_grid(n1, n2, n3)
    xc = grid.xc
    dth = math.pi / n2
    dph = 2 * math.pi / n3
    K, J, Ii = torch.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    I = _sample(Ii, J, K, ang.dir)
    Ie = TR.fill_ghosts(I, grid, ang.perm_pi2)
    NG = TR.NG
    checked = 0
    for jg in list(range(NG)) + list(range(NG + n2, 2 * NG + n2)):
        # the ghost's continued coordinate: theta = (jg - NG + 1/2) dtheta, outside [0, pi]
        th = torch.tensor((jg - NG + 0.5) * dth, dtype=F64)
        for kg in range(NG, NG + n3):
            ph = torch.tensor((kg - NG + 0.5) * dph, dtype=F64)
            for ig in range(NG, NG + n1):
                r = xc[0][ig - NG]
                want = _sample(r, th, ph, ang.dir)
                got = Ie[kg, jg, ig]
                assert (got - want).abs().max() < 1e-12, (jg, kg, ig, float((got - want).abs().max()))
                checked += 1
    assert checked == 2 * NG * n3 * n1
    # periodic ghosts in phi are the same physical cells one period away
    for kg in list(range(NG)) + list(range(NG + n3, 2 * NG + n3)):
        ph = torch.tensor((kg - NG + 0.5) * dph, dtype=F64)
        for jg in range(NG, NG + n2):
            th = xc[1][jg - NG]
            want = _sample(xc[0], th.expand(n1), ph.expand(n1), ang.dir)
            assert (Ie[kg, jg, NG:NG + n1] - want).abs().max() < 1e-12


def test_polar_ghosts_are_the_field_across_the_axis_geodesic():
    _check_polar_ghosts(GeodesicGrid(2))
    _check_polar_ghosts(GeodesicGrid(3), n2=5, n3=6)


def test_polar_ghosts_are_the_field_across_the_axis_latlong():
    _check_polar_ghosts(LatLongGrid(4, 8))


def test_polar_gas_ghosts_are_the_field_across_the_axis():
    """The gas fields' polar ghost (one layer) is the physical neighbour
    across the axis: scalars by value, the velocity's tetrad components
    rotated like the bins (pi about 2hat: u^1hat, u^3hat change sign)."""
    n1, n2, n3 = 3, 6, 8
    grid = _sph_grid(n1, n2, n3)
    xc = grid.xc
    K, J, Ii = torch.meshgrid(xc[2], xc[1], xc[0], indexing="ij")

    def phys(r, th, ph):
        er, et, ep = _frame(th, ph)
        pos = r[..., None] * er
        scal = 1.0 + 0.2 * pos[..., 0] - 0.3 * pos[..., 1] + 0.1 * pos[..., 2] ** 2
        U = torch.stack([0.1 + 0.05 * pos[..., 1], -0.2 + 0.03 * pos[..., 2], 0.07 * pos[..., 0]], -1)
        u = torch.stack([(U * ep).sum(-1), (U * er).sum(-1), (U * et).sum(-1)], -1)   # (1hat, 2hat, 3hat)
        return scal, u

    scal, u = phys(Ii, J, K)
    se = TR._gas_ghosts(scal[..., None], grid)[..., 0]
    ue = TR._gas_ghosts(u, grid, vector=True)
    dth, dph = math.pi / n2, 2 * math.pi / n3
    for jg in (0, n2 + 1):
        th = torch.tensor((jg - 0.5) * dth, dtype=F64)
        for kg in range(1, n3 + 1):
            ph = torch.tensor((kg - 0.5) * dph, dtype=F64)
            ws, wu = phys(xc[0], th.expand(n1), ph.expand(n1))
            assert (se[kg, jg, 1:n1 + 1] - ws).abs().max() < 1e-13
            assert (ue[kg, jg, 1:n1 + 1] - wu).abs().max() < 1e-13


# ---------------------------------------------------------------- CFL bound
def _ray_rate(r, th, n):
    """d n/dt of a straight ray's direction, in the spherical tetrad's
    components (1hat, 2hat, 3hat) = (phi, r, theta), flat space, c = 1.

    The direction N = n_r e_r + n_t e_t + n_p e_p of a straight ray is fixed
    while the frame turns as the ray moves along N:
      d e_r/dt = (n_t e_t + n_p e_p)/r
      d e_t/dt = (-n_t e_r + n_p cot(theta) e_p)/r
      d e_p/dt = -n_p (e_r + cot(theta) e_t)/r
    so with n_i = N . e_i:
      d n_r/dt = (n_t^2 + n_p^2)/r
      d n_t/dt = (-n_t n_r + n_p^2 cot(theta))/r
      d n_p/dt = -n_p (n_r + n_t cot(theta))/r."""
    n_p, n_r, n_t = n[..., 0], n[..., 1], n[..., 2]
    cot = math.cos(th) / math.sin(th)
    d_r = (n_t ** 2 + n_p ** 2) / r
    d_t = (-n_t * n_r + n_p ** 2 * cot) / r
    d_p = -n_p * (n_r + n_t * cot) / r
    return torch.stack([d_p, d_r, d_t], -1)


def _hand_bounds(grid, ang):
    """(spatial, angular) bounds of reading R10 from the closed forms."""
    space, angle = math.inf, math.inf
    xf = [g.numpy() for g in grid.xf]
    p, q = ang.edges[:, 0], ang.edges[:, 1]
    for j in range(grid.n[1]):
        th = 0.5 * (xf[1][j] + xf[1][j + 1])
        for i in range(grid.n[0]):
            r = 0.5 * (xf[0][i] + xf[0][i + 1])
            # coordinate speeds: dr/dt = n_r, dtheta/dt = n_t/r, dphi/dt = n_p/(r sin theta)
            sp = [ang.dir[:, 1].abs(), ang.dir[:, 2].abs() / r, ang.dir[:, 0].abs() / (r * math.sin(th))]
            for d in range(3):
                dx = xf[d][1] - xf[d][0] if d == 2 else (xf[d][i + 1] - xf[d][i] if d == 0 else xf[d][j + 1] - xf[d][j])
                m = sp[d] > 0
                space = min(space, float((dx / sp[d][m]).min()))
            V = _ray_rate(r, th, ang.edge_mid)
            w = ang.edge_len * (V * ang.edge_nrm).sum(-1).abs()
            rate = torch.zeros(ang.n_ang, dtype=F64).index_add(0, p, w).index_add(0, q, w)
            angle = min(angle, float((ang.dOmega / rate).min()))
    return space, angle


def test_angular_cfl_bound_flat_spherical_closed_form():
    ang = GeodesicGrid(2)
    # small r and coarse cells: the angular bound binds
    grid = _sph_grid(3, 4, 4, r0=1.0, r1=4.0)
    st = Setup(grid, ang)
    space, angle = _hand_bounds(grid, ang)
    assert angle < space                      # the test exercises the angular bound
    assert abs(CF.cfl_dt(st, 0.3) - 0.3 * min(space, angle)) < 1e-13 * angle
    # finer cells: the spatial bound binds, still equal to the closed form
    grid = _sph_grid(16, 16, 32, r0=1.0, r1=4.0)
    st = Setup(grid, ang)
    space, angle = _hand_bounds(grid, ang)
    assert space < angle
    assert abs(CF.cfl_dt(st, 0.3) - 0.3 * min(space, angle)) < 1e-13 * space


def test_angular_speed_is_the_straight_ray_rate():
    """The oracle's per-edge speed V . nu_e equals, up to the orientation
    convention pinned by the null-geodesic test, the turning rate of a
    straight ray's direction in the spherical frame."""
    ang = GeodesicGrid(3)
    grid = _sph_grid(2, 3, 2, r0=1.5, r1=3.0)
    st = Setup(grid, ang)
    _, s = TR.angular_speeds(st)                            # [k, j, i, e]
    for j in range(grid.n[1]):
        for i in range(grid.n[0]):
            r, th = float(grid.xc[0][i]), float(grid.xc[1][j])
            want = (_ray_rate(r, th, ang.edge_mid) * ang.edge_nrm).sum(-1)
            assert (s[0, j, i].abs() - want.abs()).abs().max() < 1e-13
            # one orientation for every edge (a fixed sign convention)
            big = want.abs() > 1e-6
            ratio = s[0, j, i][big] / want[big]
            assert (ratio.abs() - 1).abs().max() < 1e-12 and (ratio - ratio[0]).abs().max() < 1e-12
