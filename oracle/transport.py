"""Spatial grid, boundary fill, reconstruction and flux divergences.

Follows Sec. 2.2 (Eq. radiation_integral: finite-volume / finite-solid-angle
form), Sec. 2.3 (reconstruction of the primitive I per angle bin, in each
dimension separately), Sec. 2.4 (Eq. flux_space, Eq. flux_angle: upwind
fluxes, and the optical-depth weighting of the spatial fluxes) and Sec. 2.6 (angular fluxes summed over the edges of a geodesic
cell).

Layout: intensities are I[k, j, i, n] (x3, x2, x1, angle), float64.
The boundary fill builds an extended array with two ghost cells per side in
every flux dimension (Sec. 2 task list, "apply boundary conditions").
"""
import math

import numpy as np
import torch

from . import DTYPE
from . import geometry as G

NG = 3          # ghost layers: PPM reaches three cells (DC and PLM use the inner two)


class Grid:
    """Logically rectangular block of cells.

    kind, a   spacetime (see geometry.KINDS) and spin
    xf        three 1-D float64 tensors of face coordinates (n_d + 1 each)
    bc        ((lo, hi) for x1, x2, x3), each 'periodic' | 'outflow' | 'polar'
    ndim      number of dimensions that carry fluxes (the others have one cell)
    """

    def __init__(self, kind, a, xf, bc, ndim):
        self.kind, self.a = kind, float(a)
        self.xf = [torch.as_tensor(x, dtype=DTYPE) for x in xf]
        self.n = [len(x) - 1 for x in self.xf]
        self.bc = bc
        self.ndim = ndim
        for d in range(ndim, 3):
            assert self.n[d] == 1
        self.xc = [0.5 * (x[1:] + x[:-1]) for x in self.xf]

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def centres(self):
        X3, X2, X1 = torch.meshgrid(self.xc[2], self.xc[1], self.xc[0], indexing="ij")
        return torch.stack([X1, X2, X3], dim=-1)

    def polar_faces(self, d):
        """Boolean per face index along d: faces on a polar boundary."""
        m = torch.zeros(self.n[d] + 1, dtype=torch.bool)
        if self.bc[d][0] == "polar":
            m[0] = True
        if self.bc[d][1] == "polar":
            m[-1] = True
        return m


class Setup:
    """Per-cell and per-face geometric factors of Secs. 2.1-2.2 on a grid.

    All factors are evaluated at cell / face centres (coordinate midpoints):
      e, g, omega       tetrad, metric, Ricci rotation coefficients
      nup[..., n, mu]   n^mu = e^mu_A n^A, with n^0hat = 1
      nlow[..., n, mu]  n_mu
      f[..., n]         n^0 n_0  (conserved U = f I, Eq. radiation_integral)
      dV                cell volume (exact)
      fcoef[d]          Delta A_d n^d n_0 at every face along d
      fsign[d]          n^d at every face along d (upwind direction)
    """

    def __init__(self, grid, ang):
        self.grid, self.ang = grid, ang
        kind, a = grid.kind, grid.a
        X = grid.centres().reshape(-1, 3)
        e = G.batched(G.tetrad, kind, a, X)
        g = G.batched(G.metric, kind, a, X)
        om = G.batched(G.ricci_rotation, kind, a, X)
        sh = grid.shape
        self.e = e.reshape(sh + (4, 4))
        self.g = g.reshape(sh + (4, 4))
        self.omega = om.reshape(sh + (4, 4, 4))
        nhat = torch.cat([torch.ones(ang.n_ang, 1, dtype=DTYPE), ang.dir], dim=1)
        self.nhat4 = nhat
        self.nup = torch.einsum("...mA,nA->...nm", self.e, nhat)
        self.nlow = torch.einsum("...mv,...nv->...nm", self.g, self.nup)
        self.f = self.nup[..., 0] * self.nlow[..., 0]
        # exact cell volumes
        lo = torch.stack(torch.meshgrid(grid.xf[2][:-1], grid.xf[1][:-1], grid.xf[0][:-1],
                                        indexing="ij")[::-1], dim=-1)
        hi = torch.stack(torch.meshgrid(grid.xf[2][1:], grid.xf[1][1:], grid.xf[0][1:],
                                        indexing="ij")[::-1], dim=-1)
        self.dV = G.cell_volume(kind, a, lo, hi)
        # face factors
        self.fcoef, self.fsign = [], []
        for d in range(grid.ndim):
            coords = [grid.xc[0], grid.xc[1], grid.xc[2]]
            coords[d] = grid.xf[d]
            X3, X2, X1 = torch.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
            Xf = torch.stack([X1, X2, X3], dim=-1)
            polar = grid.polar_faces(d)
            # faces on the polar axis have zero area; evaluate their tetrad at
            # a regular point (the result is multiplied by zero)
            if polar.any():
                idx = [slice(None)] * 3
                idx[2 - d] = polar
                Xf = Xf.clone()
                Xf[tuple(idx) + (d,)] = grid.xc[d][0]
            fsh = Xf.shape[:-1]
            ef = G.batched(G.tetrad, kind, a, Xf.reshape(-1, 3)).reshape(fsh + (4, 4))
            gf = G.batched(G.metric, kind, a, Xf.reshape(-1, 3)).reshape(fsh + (4, 4))
            nupf = torch.einsum("...mA,nA->...nm", ef, nhat)
            n0low = torch.einsum("...v,...nv->...n", gf[..., 0, :], nupf)
            # face extents in the other two coordinates
            flo, fhi = [], []
            for dd in range(3):
                if dd == d:
                    flo.append(grid.xf[dd]); fhi.append(grid.xf[dd])
                else:
                    flo.append(grid.xf[dd][:-1]); fhi.append(grid.xf[dd][1:])
            lo = torch.stack(torch.meshgrid(flo[2], flo[1], flo[0], indexing="ij")[::-1], dim=-1)
            hi = torch.stack(torch.meshgrid(fhi[2], fhi[1], fhi[0], indexing="ij")[::-1], dim=-1)
            dA = G.face_area(kind, a, d, lo, hi)
            idx = [slice(None)] * 3
            idx[2 - d] = polar
            dA[tuple(idx)] = 0.0
            na = nupf[..., d + 1]
            self.fcoef.append(dA[..., None] * na * n0low)
            self.fsign.append(na)


# ------------------------------------------------------------ boundaries
def halo_pack(I, grid, d, side):
    """The NG layers of I next to face (d, side) of the block, as sent to the
    neighbouring block that shares the face: [NG, <the face's cells in array
    order>, Na], layer 0 adjacent to the face (the task list of Sec. 2: the
    ghost exchange between blocks)."""
    ax = 2 - d
    N = grid.n[d]
    idx = [L if side == 0 else N - 1 - L for L in range(NG)]
    return torch.stack([I.select(ax, q) for q in idx])


def fill_ghosts(I, grid, perm, halos=None):
    """Extended array with NG ghost cells per side in every flux dimension.

    periodic  ghost takes the cell one period away
    outflow   ghost copies the nearest active cell (same angle bin)
    polar     (x2 = theta only) ghost at theta -> -theta, phi -> phi + pi takes
              the active cell across the pole, with angle bin n taking bin
              perm[n] (rotation by pi about the 2-axis of the spherical
              tetrad, under which the geodesic grid is invariant)
    halo      the face is shared with another block: ghost layer L (0 next to
              the face) is halos[(d, side)][L], the neighbour's halo_pack of
              the same face
    """
    N1, N2, N3 = grid.n
    Na = I.shape[-1]
    Ie = torch.zeros((N3 + 2 * NG, N2 + 2 * NG, N1 + 2 * NG, Na), dtype=I.dtype)
    act = (slice(NG, NG + N3), slice(NG, NG + N2), slice(NG, NG + N1))
    Ie[act] = I
    for d in range(grid.ndim):
        ax = 2 - d                       # array dimension of coordinate d
        N = grid.n[d]
        for side in (0, 1):
            kind = grid.bc[d][side]
            for gidx in range(NG):       # ghost layer 0 is adjacent to the boundary
                if side == 0:
                    gpos = NG - 1 - gidx
                else:
                    gpos = NG + N + gidx
                if kind == "periodic":
                    src = (N - 1 - gidx) if side == 0 else gidx
                    shift, pm = 0, None
                elif kind == "outflow":
                    src = 0 if side == 0 else N - 1
                    shift, pm = 0, None
                elif kind == "polar":
                    assert d == 1
                    src = gidx if side == 0 else N - 1 - gidx
                    shift, pm = N3 // 2, perm
                elif kind == "halo":
                    sl_dst = list(act)
                    sl_dst[ax] = gpos
                    Ie[tuple(sl_dst)] = halos[(d, side)][gidx]
                    continue
                else:
                    raise ValueError(kind)
                sl_dst = list(act)
                sl_dst[ax] = slice(gpos, gpos + 1)
                sl_src = list(act)
                sl_src[ax] = slice(NG + src, NG + src + 1)
                vals = Ie[tuple(sl_src)].clone()
                if shift:
                    vals = torch.roll(vals, shifts=-shift, dims=0)
                if pm is not None:
                    vals = vals[..., pm]
                Ie[tuple(sl_dst)] = vals
    return Ie


# ------------------------------------------------------- reconstruction
def van_leer(dl, dr):
    """Harmonic-mean slope of van Leer (1974): 2 dl dr / (dl + dr) if dl dr > 0."""
    prod = dl * dr
    pos = prod > 0.0
    den = torch.where(pos, dl + dr, torch.ones_like(dl))
    return torch.where(pos, 2.0 * prod / den, torch.zeros_like(dl))


def ppm_edges(line, ax):
    """Monotonised parabola edge values (aL, aR) of every cell of a line (the
    piecewise parabolic method of Colella & Woodward 1984, cited in Sec. 2.3,
    on a uniform index grid): van Leer / monotonised-central limited slopes,
    fourth-order interface values from them, then the two monotonicity
    constraints (flatten at local extrema; pull the far edge in when the
    parabola would overshoot).  Returns arrays for cells 2 .. L-3 of the line."""
    L = line.shape[ax]

    def take(lo, hi, x=line):
        s = [slice(None)] * x.dim()
        s[ax] = slice(lo, hi)
        return x[tuple(s)]

    am, a0, ap = take(0, L - 2), take(1, L - 1), take(2, L)          # cells 1 .. L-2
    dc = 0.5 * (ap - am)
    dl, dr = a0 - am, ap - a0
    mag = torch.minimum(dc.abs(), torch.minimum(2.0 * dl.abs(), 2.0 * dr.abs()))
    slope = torch.where(dl * dr > 0.0, torch.sign(dc) * mag, torch.zeros_like(dc))
    # interface e between cells e-1 and e, e = 2 .. L-2 (slope index = cell - 1)
    edge = 0.5 * (take(1, L - 2) + take(2, L - 1)) - (take(1, L - 2, slope) - take(0, L - 3, slope)) / 6.0
    a = take(2, L - 2)                                                # cells 2 .. L-3
    aL, aR = take(0, L - 4, edge), take(1, L - 3, edge)
    flat = (aR - a) * (a - aL) <= 0.0
    aL, aR = torch.where(flat, a, aL), torch.where(flat, a, aR)
    dlr = aR - aL
    six = dlr * (a - 0.5 * (aL + aR))
    over_l = six > dlr * dlr / 6.0
    over_r = -dlr * dlr / 6.0 > six
    aL = torch.where(over_l, 3.0 * a - 2.0 * aR, aL)
    aR = torch.where(over_r & ~over_l, 3.0 * a - 2.0 * aL, aR)
    return aL, aR


def face_states(Ie, grid, d, recon):
    """Left/right states of I at the n_d + 1 faces along coordinate d (Sec. 2.3)."""
    ax = 2 - d
    N = grid.n[d]
    sl = [slice(NG, NG + grid.n[2]), slice(NG, NG + grid.n[1]), slice(NG, NG + grid.n[0])]
    sl[ax] = slice(None)
    line = Ie[tuple(sl)]                    # all NG + N + NG cells along ax

    def take(lo, hi):
        s = [slice(None)] * 4
        s[ax] = slice(lo, hi)
        return line[tuple(s)]

    # face f (0..N) sits between extended cells f + NG - 1 and f + NG
    IL = take(NG - 1, NG + N)
    IR = take(NG, NG + N + 1)
    if recon == "dc":
        return IL, IR
    if recon == "ppm":
        aL, aR = ppm_edges(line, ax)                    # cells 2 .. N + 2 NG - 3
        s = [slice(None)] * 4
        s[ax] = slice(NG - 3, NG - 3 + N + 1)          # right edges of cells NG-1 .. NG+N-1
        left = aR[tuple(s)]
        s[ax] = slice(NG - 2, NG - 2 + N + 1)          # left edges of cells NG .. NG+N
        right = aL[tuple(s)]
        return left, right
    dL = take(1, NG + N + 1) - take(0, NG + N)          # I_c - I_{c-1}, c = 1..N+NG
    dR = take(2, NG + N + 2) - take(1, NG + N + 1)      # I_{c+1} - I_c
    slope = van_leer(dL, dR)                            # at extended cells 1..N+NG
    s = [slice(None)] * 4
    s[ax] = slice(NG - 2, NG - 2 + N + 1)
    sL = slope[tuple(s)]                                # cells NG-1 .. NG+N-1
    s[ax] = slice(NG - 1, NG - 1 + N + 1)
    sR = slope[tuple(s)]                                # cells NG .. NG+N
    return IL + 0.5 * sL, IR - 0.5 * sR


def _gas_ghosts(field, grid, vector=False):
    """Gas field [n3, n2, n1, ...] extended by one ghost layer per side in every
    flux dimension: periodic wrap, outflow copy, polar mirror (the cell across
    the pole, at phi + pi; a tetrad-frame vector field [..., 3] (vector=True)
    is rotated like the angle bins, by pi about 2hat, so u^1hat and u^3hat
    change sign).  Polar faces have zero area, so a polar ghost's value never
    reaches a flux."""
    N1, N2, N3 = grid.n
    ext = field
    for d in range(grid.ndim):
        ax = 2 - d
        N = grid.n[d]
        parts = []
        for side in (0, 1):
            kind = grid.bc[d][side]
            if kind == "periodic":
                src = N - 1 if side == 0 else 0
            else:                       # outflow copy, polar mirror
                src = 0 if side == 0 else N - 1
            v = ext.narrow(ax, src, 1)
            if kind == "polar":
                v = torch.roll(v, shifts=-(N3 // 2), dims=0)
                if vector:
                    v = v * torch.tensor([-1.0, 1.0, -1.0], dtype=v.dtype)
            parts.append(v)
        ext = torch.cat([parts[0], ext, parts[1]], dim=ax)
    return ext


def tau_weights(setup, gas, dt, C):
    """Optical-depth weighting of the spatial fluxes (Sec. 2.4, after Eq.
    flux_space).  Per flux dimension, returns the factors (1 - g_L + g,
    1 - g_R + g) at every face and bin, applied to the left / right upwind
    state:
        u^a, alpha_E = alpha_a + alpha_s   averaged to the face from its two cells
        tau = C alpha_E dt / u^0hat        (u^0hat of the face velocity)
        f   = -expm1(-tau^2)
        g_X = -f (1 + 1 / n^0bar_X),  n^0bar_X = u^0hat_X - u_ahat,X n^ahat
              (X = L, R: the cells on the lesser / greater side)
        g   = (g_L + g_R) / 2
    C = 0 gives f = 0 and both factors 1 (the free-streaming flux)."""
    grid = setup.grid
    u = gas["u"]
    aE = gas["alpha_a"] + gas["alpha_s"]
    ue = _gas_ghosts(u, grid, vector=True)          # [.., 3]
    ae = _gas_ghosts(aE[..., None], grid)[..., 0]
    out = []
    for d in range(grid.ndim):
        ax = 2 - d
        N = grid.n[d]
        off = [1 if dd < grid.ndim else 0 for dd in range(3)]      # ghost layers per dimension
        sl = [slice(off[2], off[2] + grid.n[2]), slice(off[1], off[1] + grid.n[1]),
              slice(off[0], off[0] + grid.n[0])]
        sl[ax] = slice(None)
        uline, aline = ue[tuple(sl)], ae[tuple(sl)]    # cells -1 .. N along ax
        uL, uR = uline.narrow(ax, 0, N + 1), uline.narrow(ax, 1, N + 1)
        aL, aR = aline.narrow(ax, 0, N + 1), aline.narrow(ax, 1, N + 1)
        uF = 0.5 * (uL + uR)
        aF = 0.5 * (aL + aR)
        u0F = torch.sqrt(1.0 + (uF * uF).sum(-1))
        tau = C * aF * dt / u0F
        f = -torch.expm1(-tau * tau)
        nbarL = torch.sqrt(1.0 + (uL * uL).sum(-1))[..., None] - uL @ setup.ang.dir.T
        nbarR = torch.sqrt(1.0 + (uR * uR).sum(-1))[..., None] - uR @ setup.ang.dir.T
        gL = -f[..., None] * (1.0 + 1.0 / nbarL)
        gR = -f[..., None] * (1.0 + 1.0 / nbarR)
        g = 0.5 * (gL + gR)
        out.append((1.0 - gL + g, 1.0 - gR + g))
    return out


def spatial_divergence(Ie, setup, recon, tau=None):
    """(1/dV) sum_d [dA n^d n_0 I_upwind]^+_- (Eq. flux_space, Eq. radiation_integral);
    with tau (from tau_weights) the upwind states carry the optical-depth
    factors of Sec. 2.4."""
    grid = setup.grid
    div = torch.zeros(grid.shape + (Ie.shape[-1],), dtype=Ie.dtype)
    for d in range(grid.ndim):
        ax = 2 - d
        IL, IR = face_states(Ie, grid, d, recon)
        if tau is not None:
            IL, IR = IL * tau[d][0], IR * tau[d][1]
        up = torch.where(setup.fsign[d] < 0.0, IR, IL)     # tie -> left state
        F = setup.fcoef[d] * up
        N = grid.n[d]
        hi = F.narrow(ax, 1, N)
        lo = F.narrow(ax, 0, N)
        div = div + (hi - lo)
    return div / setup.dV[..., None]


def angular_speeds(setup):
    """Per cell and edge: l_e * (V . nu_e) * n_0(n_e)  (Eq. flux_angle, Sec. 2.6).

    V is the angular velocity field on the unit sphere implied by the
    symbols n^zeta, n^psi (the tangent part of -omega^i_{AB} n^A n^B); it is
    evaluated at the edge midpoint n_e and projected on the edge normal nu_e
    (from cell p to cell q).  n_0 uses the cell-centre tetrad at direction n_e.
    """
    ang = setup.ang
    ne4 = torch.cat([torch.ones(len(ang.edge_len), 1, dtype=DTYPE), ang.edge_mid], dim=1)
    Q = torch.einsum("...CAB,eA,eB->...eC", setup.omega, ne4, ne4)
    V = -(Q[..., 1:] - ang.edge_mid * Q[..., :1])
    s = (V * ang.edge_nrm).sum(-1)
    n0 = torch.einsum("...v,...vA,eA->...e", setup.g[..., 0, :], setup.e, ne4)
    return ang.edge_len * s * n0, s


def mapr_stencils(ang):
    """Per cell c of a geodesic grid, the geometry of its minimum-angle plane
    reconstruction: its neighbours in cyclic order around n_c, their
    gnomonic coordinates x = (v . t1, v . t2) / (v . n_c) in the tangent
    plane at n_c (t1, t2 any orthonormal pair normal to n_c), and the
    gnomonic coordinates of the midpoints of its sides.  Returns a list of
    (neighbours, X [K, 2], {neighbour: (side, x_side)})."""
    if getattr(ang, "_mapr", None) is not None:
        return ang._mapr
    dirs = ang.dir.numpy()
    mids = ang.edge_mid.numpy()
    side = {}
    for e, (p, q) in enumerate(ang.edges.tolist()):
        side[(p, q)] = e
        side[(q, p)] = e
    out = []
    for c in range(ang.n_ang):
        n = dirs[c]
        t1 = np.cross(n, [0.3, 0.5, 0.7])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(n, t1)

        def gn(v):
            return np.array([v @ t1, v @ t2]) / (v @ n)

        nb = sorted(ang.nbr[c], key=lambda m: math.atan2(dirs[m] @ t2, dirs[m] @ t1))
        X = np.array([gn(dirs[m]) for m in nb])
        xs = {m: (side[(c, m)], gn(mids[side[(c, m)]])) for m in nb}
        out.append((nb, X, xs))
    ang._mapr = out
    return out


def mapr_face_values(I, ang):
    """Upwind candidates at every side p | q by minimum-angle plane
    reconstruction (MAPR), which the paper names for geodesic grids (Sec.
    2.6) without stating it.  Reading: around cell c every two cyclically
    adjacent neighbours a, b fix a plane through (0, I_c), (x_a, I_a),
    (x_b, I_b) in c's gnomonic tangent plane, i.e. a gradient g with
    g . x_a = I_a - I_c and g . x_b = I_b - I_c; the least inclined plane
    (smallest |g|; the first in cyclic order on a tie) is kept, and c's value
    at a side is I_c + g . x_side."""
    st = mapr_stencils(ang)
    n_edge = ang.edges.shape[0]
    vals = [[None, None] for _ in range(n_edge)]
    for c, (nb, X, xs) in enumerate(st):
        Ic = I[..., c]
        K = len(nb)
        best_g = best_q = None
        for a in range(K):
            b = (a + 1) % K
            M = torch.tensor(np.array([X[a], X[b]]), dtype=I.dtype)
            d = torch.stack([I[..., nb[a]] - Ic, I[..., nb[b]] - Ic], -1)
            g = torch.linalg.solve(M, d.unsqueeze(-1)).squeeze(-1)      # M g = d
            q = (g * g).sum(-1)
            if best_g is None:
                best_g, best_q = g, q
            else:
                take = q < best_q
                best_g = torch.where(take[..., None], g, best_g)
                best_q = torch.where(take, q, best_q)
        for m in nb:
            e, xe = xs[m]
            v = Ic + (best_g * torch.tensor(xe, dtype=I.dtype)).sum(-1)
            vals[e][0 if int(ang.edges[e, 0]) == c else 1] = v
    Fp = torch.stack([v[0] for v in vals], -1)
    Fq = torch.stack([v[1] for v in vals], -1)
    return Fp, Fq


def angular_face_values(I, ang, recon_ang="dc"):
    """Upwind candidates at every side p | q: (value from p, value from q).

    DC: the cell values.  PLM (latitude-longitude grids, Sec. 2.6): the
    spatial reconstruction applied along the line through p and q, i.e.
    I_p + van_leer(I_p - I_behind, I_q - I_p) / 2 from p and
    I_q + van_leer(I_q - I_beyond, I_p - I_q) / 2 from q.  MAPR (geodesic
    grids): mapr_face_values."""
    p, q = ang.edges[:, 0], ang.edges[:, 1]
    Ip, Iq = I[..., p], I[..., q]
    if recon_ang == "dc":
        return Ip, Iq
    if recon_ang == "mapr":
        if hasattr(ang, "edge_line"):
            raise ValueError("MAPR is defined here for geodesic grids")
        return mapr_face_values(I, ang)
    if recon_ang != "plm" or not hasattr(ang, "edge_line"):
        raise ValueError("angular PLM needs a latitude-longitude grid")
    Ib, If = I[..., ang.edge_line[:, 0]], I[..., ang.edge_line[:, 1]]
    return Ip + 0.5 * van_leer(Ip - Ib, Iq - Ip), Iq + 0.5 * van_leer(Iq - If, Ip - Iq)


def angular_divergence(I, setup, recon_ang="dc"):
    """(1/dOmega_p) sum over the edges of p of the outgoing upwind flux."""
    ang = setup.ang
    coef, s = angular_speeds(setup)
    p, q = ang.edges[:, 0], ang.edges[:, 1]
    Fp, Fq = angular_face_values(I, ang, recon_ang)
    F = coef * torch.where(s < 0.0, Fq, Fp)            # tie -> p side
    div = torch.zeros_like(I)
    div = div.index_add(-1, p, F / ang.dOmega[p])
    div = div.index_add(-1, q, -F / ang.dOmega[q])
    return div
