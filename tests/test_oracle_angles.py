"""Pins of the oracle's geodesic angle grid (Sec. 2.6) against facts that do
not depend on its code: counts fixed by the construction, exact symmetry
values, an independent area formula and the divergence theorem on the sphere."""
import math

import numpy as np
import pytest
import torch

from oracle.angles import GeodesicGrid


@pytest.fixture(scope="module", params=[1, 2, 3, 4, 6])
def grid(request):
    return GeodesicGrid(request.param)


def test_counts_and_topology(grid):
    N = grid.N
    # Sec. 2.6: 10 N^2 + 2 cells, 12 of them pentagons, the rest hexagons
    assert grid.n_ang == 10 * N * N + 2
    deg = [len(x) for x in grid.nbr]
    assert deg.count(5) == 12 and deg.count(6) == grid.n_ang - 12
    # Euler characteristic of the dual polygon mesh: V - E + F = 2
    assert grid.n_corner - len(grid.edges) + grid.n_ang == 2
    for p, ns in enumerate(grid.nbr):
        for q in ns:
            assert p in grid.nbr[q]


def test_solid_angles_sum_to_4pi(grid):
    assert abs(float(grid.dOmega.sum()) - 4 * math.pi) < 1e-13


def test_level1_pentagons_are_pi_over_3():
    g = GeodesicGrid(1)
    assert torch.allclose(g.dOmega, torch.full((12,), math.pi / 3, dtype=torch.float64), atol=1e-15, rtol=0)


def _girard_area(centre, corners):
    """Spherical excess from interior angles (Girard), independent of the fan."""
    c = np.asarray(centre)
    e1 = np.cross(c, [0.3, 0.5, 0.7]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    cs = sorted(corners, key=lambda x: math.atan2(np.dot(x, e2), np.dot(x, e1)))
    m = len(cs)
    tot = 0.0
    for k in range(m):
        p, v, nx = cs[k - 1], cs[k], cs[(k + 1) % m]
        t1 = p - np.dot(p, v) * v
        t2 = nx - np.dot(nx, v) * v
        tot += math.atan2(np.linalg.norm(np.cross(t1, t2)), np.dot(t1, t2))
    return tot - (m - 2) * math.pi


def test_area_matches_girard(grid):
    for v in range(0, grid.n_ang, max(1, grid.n_ang // 17)):
        corners = [grid.corners[t] for t in grid.tri_of_vertex[v]]
        ref = _girard_area(grid.dir[v].numpy(), corners)
        assert abs(ref - float(grid.dOmega[v])) < 1e-12


def test_icosahedral_symmetry_moments(grid):
    # first and second moments of an icosahedrally symmetric quadrature
    m1 = (grid.dir * grid.dOmega[:, None]).sum(0)
    m2 = torch.einsum("ni,nj,n->ij", grid.dir, grid.dir, grid.dOmega)
    assert m1.abs().max() < 1e-14
    assert (m2 - 4 * math.pi / 3 * torch.eye(3, dtype=torch.float64)).abs().max() < 1e-13


def test_pi_rotation_about_axis2_is_a_symmetry(grid):
    perm = grid.perm_pi2
    assert grid.perm_err < 1e-14
    assert sorted(perm.tolist()) == list(range(grid.n_ang))
    assert torch.equal(perm[perm], torch.arange(grid.n_ang))
    R = torch.tensor([-1.0, 1.0, -1.0], dtype=torch.float64)
    assert (grid.dir[perm] - grid.dir * R).abs().max() < 1e-14
    assert (grid.dOmega[perm] - grid.dOmega).abs().max() < 1e-14


def test_edges_geometry(grid):
    # normals are unit, tangent at the midpoint, and point from p to q
    nu, mid = grid.edge_nrm, grid.edge_mid
    assert ((nu * nu).sum(-1) - 1).abs().max() < 1e-14
    assert (nu * mid).sum(-1).abs().max() < 1e-14
    p, q = grid.edges[:, 0], grid.edges[:, 1]
    assert ((grid.dir[q] - grid.dir[p]) * nu).sum(-1).min() > 0
    # the polygon perimeters close: sum of edge lengths per cell ~ sqrt of area
    per = torch.zeros(grid.n_ang, dtype=torch.float64).index_add(0, p, grid.edge_len).index_add(0, q, grid.edge_len)
    assert (per ** 2 / grid.dOmega).max() < 16.0


def _edge_flux(grid, field):
    """Sum over the edges of every cell of l_e w(n_e) . nu_e (outward)."""
    w = field(grid.edge_mid)
    F = grid.edge_len * (w * grid.edge_nrm).sum(-1)
    p, q = grid.edges[:, 0], grid.edges[:, 1]
    return torch.zeros(grid.n_ang, dtype=torch.float64).index_add(0, p, F).index_add(0, q, -F)


def test_divergence_theorem_on_sphere():
    """For w = k - (n.k) n, div_sphere w = -2 n.k, and w.nu is constant along a
    great-circle edge, so the edge sums are exact integrals; their ratio to
    the cell area converges to the pointwise divergence as the grid refines.
    A rigid rotation (zero divergence) leaves a residual that also shrinks."""
    k = torch.tensor([0.3, -0.5, 0.8], dtype=torch.float64)
    om = torch.tensor([0.2, 0.7, -0.4], dtype=torch.float64)
    errs, rots = [], []
    for N in (2, 4, 8):
        g = GeodesicGrid(N)
        flux = _edge_flux(g, lambda n: k - (n @ k)[:, None] * n)
        exact = -2.0 * (g.dir @ k) * g.dOmega
        errs.append(float(((flux - exact).abs() / g.dOmega).max()))
        rot = _edge_flux(g, lambda n: torch.cross(om.expand_as(n), n, dim=-1))
        rots.append(float((rot.abs() / g.dOmega).max()))
        # conservation: every edge flux leaves one cell and enters another
        assert abs(float(flux.sum())) < 1e-13
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.012
    assert rots[0] < 1e-14 and rots[2] < rots[1] < 2e-3
