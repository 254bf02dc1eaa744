"""Pins of the oracle's latitude-longitude angle grid (Sec. 2.6): equal solid
angles summing to 4 pi, the second moment of the directions, the pi rotation
about the 2-axis, edge geometry, the divergence theorem on the sphere, and
the paper's statement that for N_psi = 2 N_zeta the cells touching a pole
have a short-to-long side ratio of about pi / N_zeta."""
import math

import pytest
import torch

from oracle.angles import LatLongGrid

F64 = torch.float64


def _edge_flux(grid, field):
    """Sum over the edges of every cell of l_e w(n_e) . nu_e (outward)."""
    w = field(grid.edge_mid)
    F = grid.edge_len * (w * grid.edge_nrm).sum(-1)
    p, q = grid.edges[:, 0], grid.edges[:, 1]
    return torch.zeros(grid.n_ang, dtype=F64).index_add(0, p, F).index_add(0, q, -F)


@pytest.mark.parametrize("nz,npsi", [(1, 4), (3, 4), (4, 8), (9, 18), (6, 10)])
def test_counts_solid_angles_and_topology(nz, npsi):
    g = LatLongGrid(nz, npsi)
    assert g.n_ang == nz * npsi
    assert abs(float(g.dOmega.sum()) - 4 * math.pi) < 1e-13
    assert float((g.dOmega - 4 * math.pi / (nz * npsi)).abs().max()) < 1e-15
    assert float(((g.dir * g.dir).sum(-1) - 1).abs().max()) < 1e-15
    # meridians between all sectors of a band, latitude lines between bands
    assert len(g.edges) == nz * npsi + (nz - 1) * npsi
    deg = [len(x) for x in g.nbr]
    assert all(d == (2 if nz == 1 else (3 if (n < npsi or n >= g.n_ang - npsi) else 4)) for n, d in enumerate(deg))
    for p, ns in enumerate(g.nbr):
        for q in ns:
            assert p in g.nbr[q]


@pytest.mark.parametrize("nz,npsi", [(1, 4), (3, 4), (4, 8), (9, 18)])
def test_pi_rotation_about_axis2_is_a_permutation(nz, npsi):
    g = LatLongGrid(nz, npsi)
    assert sorted(g.perm_pi2.tolist()) == list(range(g.n_ang))
    rot = g.dir * torch.tensor([-1.0, 1.0, -1.0], dtype=F64)
    assert float((g.dir[g.perm_pi2] - rot).abs().max()) < 4e-15


def test_direction_moments():
    """sum n dOmega = 0 by symmetry; sum n n dOmega -> (4 pi / 3) 1 at second
    order under refinement (the directions are cell points, not centroids)."""
    errs = []
    for nz in (4, 8, 16):
        g = LatLongGrid(nz, 2 * nz)
        assert float((g.dir * g.dOmega[:, None]).sum(0).abs().max()) < 1e-14
        M = torch.einsum("na,nb,n->ab", g.dir, g.dir, g.dOmega)
        off = M - torch.diag(torch.diagonal(M))
        assert float(off.abs().max()) < 1e-14
        errs.append(float((torch.diagonal(M) - 4 * math.pi / 3).abs().max()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("nz,npsi", [(3, 4), (4, 8), (9, 18)])
def test_edges_geometry(nz, npsi):
    g = LatLongGrid(nz, npsi)
    nu, mid = g.edge_nrm, g.edge_mid
    assert float(((nu * nu).sum(-1) - 1).abs().max()) < 1e-14
    assert float((nu * mid).sum(-1).abs().max()) < 1e-15
    p, q = g.edges[:, 0], g.edges[:, 1]
    assert float(((g.dir[q] - g.dir[p]) * nu).sum(-1).min()) > 0
    # the sides of a band's cells add up to the band's two latitude circles
    # and 2 N_psi meridian arcs
    dz = torch.tensor([math.acos(1 - 2 * (i + 1) / nz) - math.acos(1 - 2 * i / nz) for i in range(nz)], dtype=F64)
    per = torch.zeros(g.n_ang, dtype=F64).index_add(0, p, g.edge_len).index_add(0, q, g.edge_len)
    band = per.view(nz, npsi).sum(-1)
    sinb = torch.tensor([math.sqrt(max(0.0, 1 - (1 - 2 * i / nz) ** 2)) for i in range(nz + 1)], dtype=F64)
    ref = 2 * math.pi * (sinb[:-1] + sinb[1:]) + 2 * npsi * dz
    assert float((band - ref).abs().max()) < 1e-12


def test_divergence_theorem_on_sphere():
    """For w = k - (n.k) n, div_sphere w = -2 n.k.  On meridian sides w.nu is
    constant and the midpoint rule is exact; on latitude sides it is a
    one-point rule.  The cell sums over the cell area converge to the
    pointwise divergence; a rigid rotation about the pole axis gives zero
    exactly, about another axis a residual that shrinks."""
    k = torch.tensor([0.3, -0.5, 0.8], dtype=F64)
    om = torch.tensor([0.2, 0.7, -0.4], dtype=F64)
    ez = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    errs, rots = [], []
    for nz in (4, 8, 16, 32):
        g = LatLongGrid(nz, 2 * nz)
        flux = _edge_flux(g, lambda n: k - (n @ k)[:, None] * n)
        exact = -2.0 * (g.dir @ k) * g.dOmega
        errs.append(float(((flux - exact).abs() / g.dOmega).mean()))
        assert abs(float(flux.sum())) < 1e-13
        zrot = _edge_flux(g, lambda n: torch.cross(ez.expand_as(n), n, dim=-1))
        assert float((zrot.abs() / g.dOmega).max()) < 1e-13
        rot = _edge_flux(g, lambda n: torch.cross(om.expand_as(n), n, dim=-1))
        rots.append(float((rot.abs() / g.dOmega).mean()))
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 0.02
    assert rots[0] > rots[1] > rots[2] > rots[3]


def test_polar_cells_side_ratio_is_pi_over_n_zeta():
    """Sec. 2.6: with N_psi = 2 N_zeta the spherical triangles at a pole have
    a short-to-long side ratio that scales as pi / N_zeta."""
    ratios = []
    for nz in (16, 64, 256):
        g = LatLongGrid(nz, 2 * nz)
        p, q = g.edges[:, 0], g.edges[:, 1]
        cap = 0                                   # a cell of the northern cap
        sides = g.edge_len[(p == cap) | (q == cap)]
        ratios.append(float(sides.min() / sides.max()) * nz / math.pi)
    assert abs(ratios[-1] - 1.0) < 3e-3           # sin(zeta_1) / zeta_1 = 1 - 2 / (3 N_zeta) + ...
    assert abs(ratios[0] - 1.0) > abs(ratios[1] - 1.0) > abs(ratios[2] - 1.0)


@pytest.mark.parametrize("nz,npsi", [(2, 4), (3, 8), (6, 12)])
def test_line_neighbours(nz, npsi):
    """Behind p and beyond q lie on the line through p and q: for a meridian
    side the band's next sectors; for a latitude side the sector's next
    bands, continued across a pole into sector psi + pi of the same band."""
    g = LatLongGrid(nz, npsi)
    for (p, q), (b, f) in zip(g.edges.tolist(), g.edge_line.tolist()):
        ip, jp, iq, jq = p // npsi, p % npsi, q // npsi, q % npsi
        ib, jb, i_f, jf = b // npsi, b % npsi, f // npsi, f % npsi
        if ip == iq:                                     # meridian: psi line in one band
            d = (jq - jp) % npsi                         # +1 or -1 (wrap)
            assert d in (1, npsi - 1)
            step = 1 if d == 1 else -1
            assert ib == ip and jb == (jp - step) % npsi
            assert i_f == iq and jf == (jq + step) % npsi
        else:                                            # latitude: zeta line of one sector
            assert jp == jq and iq == ip + 1
            if ip > 0:
                assert (ib, jb) == (ip - 1, jp)
            else:                                        # across the north pole
                assert (ib, jb) == (0, (jp + npsi // 2) % npsi)
            if iq < nz - 1:
                assert (i_f, jf) == (iq + 1, jq)
            else:                                        # across the south pole
                assert (i_f, jf) == (nz - 1, (jq + npsi // 2) % npsi)


def test_plm_face_values_are_exact_for_linear_data():
    """Away from the poles and the psi wrap, data linear in the band and
    sector indices are reconstructed exactly at the sides (the midpoint of
    the two cell values), as the spatial PLM does."""
    from oracle.transport import angular_face_values
    nz, npsi = 8, 16
    g = LatLongGrid(nz, npsi)
    i, j = torch.arange(nz).repeat_interleave(npsi), torch.arange(npsi).repeat(nz)
    I = (3.0 + 0.25 * i + 0.125 * j).to(F64)
    Fp, Fq = angular_face_values(I, g, "plm")
    p, q = g.edges[:, 0], g.edges[:, 1]
    b, f = g.edge_line[:, 0], g.edge_line[:, 1]
    # interior lines: no wrap in psi, no pole crossing
    ok = ((j[p] - j[b]).abs() <= 1) & ((j[f] - j[q]).abs() <= 1) & ((j[q] - j[p]).abs() <= 1)
    ok &= ((i[p] - i[b]) == (i[q] - i[p])) & ((i[f] - i[q]) == (i[q] - i[p]))
    assert int(ok.sum()) > len(p) // 2
    mid = 0.5 * (I[p] + I[q])
    assert float((Fp - mid)[ok].abs().max()) < 1e-14
    assert float((Fq - mid)[ok].abs().max()) < 1e-14


def _rotation_divergence_error(nz, recon, axis):
    """L1 error (over the sphere) of the discrete divergence of v f with the
    rigid rotation v = axis x n and f = 1 + 0.5 n.k, whose exact divergence
    is v . grad f = 0.5 (axis x n) . k."""
    from oracle.transport import angular_face_values
    g = LatLongGrid(nz, 2 * nz)
    k = torch.tensor([0.3, -0.5, 0.6], dtype=F64)
    f = 1.0 + 0.5 * (g.dir @ k)
    vel = torch.cross(axis.expand_as(g.edge_mid), g.edge_mid, dim=-1)
    s = (vel * g.edge_nrm).sum(-1)
    Fp, Fq = angular_face_values(f, g, recon)
    F = g.edge_len * s * torch.where(s < 0.0, Fq, Fp)
    p, q = g.edges[:, 0], g.edges[:, 1]
    div = torch.zeros(g.n_ang, dtype=F64).index_add(0, p, F).index_add(0, q, -F) / g.dOmega
    exact = 0.5 * (torch.cross(axis.expand_as(g.dir), g.dir, dim=-1) @ k)
    return float(((div - exact).abs() * g.dOmega).sum())


def test_plm_beats_dc_and_converges_faster_along_the_bands():
    """Rotation about the pole axis moves intensity along the bands (psi
    lines, uniform in index): the DC error halves with each refinement,
    the PLM error falls about 13-fold over two.  Rotation about the 1-axis
    crosses latitude sides and the poles, where the bands are uniform in
    cos(zeta) rather than zeta (a mapping singular at the poles), so the
    index-space PLM stays first order there, with a smaller constant than
    DC at every resolution."""
    z, x = torch.tensor([0.0, 0.0, 1.0], dtype=F64), torch.tensor([1.0, 0.0, 0.0], dtype=F64)
    dc = [_rotation_divergence_error(n, "dc", z) for n in (8, 16, 32)]
    pl = [_rotation_divergence_error(n, "plm", z) for n in (8, 16, 32)]
    assert 1.6 < dc[0] / dc[1] < 2.5 and 1.6 < dc[1] / dc[2] < 2.5
    assert pl[0] / pl[2] > 9.0 and pl[2] < 0.1 * dc[2]
    dcx = [_rotation_divergence_error(n, "dc", x) for n in (8, 16, 32)]
    plx = [_rotation_divergence_error(n, "plm", x) for n in (8, 16, 32)]
    assert plx[0] > plx[1] > plx[2]
    assert all(a < 0.7 * b for a, b in zip(plx, dcx))
