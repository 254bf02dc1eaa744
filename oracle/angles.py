"""Geodesic angle grid (Sec. 2.6, the three-step construction of Wang 2011).

Reading of the construction (it is stated only in words):
  * an icosahedron with one vertex on the +3 axis (the figure of angular
    grids puts a pentagon at the pole); the upper ring of five vertices sits
    at azimuths 2*pi*k/5, the lower ring at 2*pi*k/5 + pi/5, which makes the
    +2 axis one of the icosahedron's two-fold axes;
  * every face is cut *flat* into N^2 equal triangles (barycentric lattice
    a + b + c = N);
  * the radiation directions (cell centres) are the lattice vertices
    projected onto the unit sphere; there are 10 N^2 + 2 of them;
  * the cell around a vertex is the spherical polygon whose corners are the
    projected centroids of the flat lattice triangles touching the vertex,
    joined by great-circle arcs (the "spherical geodesic edges").

Everything here is plain float64 and built by brute force: vertices are
deduplicated by position, polygon corners are found by scanning the triangle
list, and areas use L'Huilier's theorem on a fan of spherical triangles.
"""
import math

import numpy as np
import torch

from . import DTYPE


def icosahedron():
    """12 unit vertices and 20 faces, vertex 0 at +z, vertex 11 at -z."""
    h = 1.0 / math.sqrt(5.0)          # height of the two rings
    r = 2.0 / math.sqrt(5.0)          # radius of the two rings
    v = [(0.0, 0.0, 1.0)]
    for k in range(5):
        psi = 2.0 * math.pi * k / 5.0
        v.append((r * math.cos(psi), r * math.sin(psi), h))
    for k in range(5):
        psi = 2.0 * math.pi * k / 5.0 + math.pi / 5.0
        v.append((r * math.cos(psi), r * math.sin(psi), -h))
    v.append((0.0, 0.0, -1.0))
    U = [1 + k for k in range(5)]
    L = [6 + k for k in range(5)]
    faces = []
    for k in range(5):
        k1 = (k + 1) % 5
        faces.append((0, U[k], U[k1]))          # top cap
        faces.append((U[k], L[k], U[k1]))       # upper band
        faces.append((L[k], L[k1], U[k1]))      # lower band
        faces.append((11, L[k1], L[k]))         # bottom cap
    return np.array(v, dtype=np.float64), faces


def _lhuilier(a, b, c):
    """Area of the spherical triangle with unit vertices a, b, c."""
    def arc(x, y):
        return math.atan2(np.linalg.norm(np.cross(x, y)), float(np.dot(x, y)))
    A, B, C = arc(b, c), arc(c, a), arc(a, b)
    s = 0.5 * (A + B + C)
    t = (math.tan(0.5 * s) * math.tan(0.5 * (s - A))
         * math.tan(0.5 * (s - B)) * math.tan(0.5 * (s - C)))
    return 4.0 * math.atan(math.sqrt(max(t, 0.0)))


class GeodesicGrid:
    """Angle grid of level N (Sec. 2.6).

    Attributes (float64 torch tensors unless noted)
      n_ang      10 N^2 + 2
      dir        [n_ang, 3]  unit direction n^i-hat of every cell centre
      dOmega     [n_ang]     solid angle of every cell
      nbr        list of neighbour lists (python ints)
      edges      [n_edge, 2] (p, q) with p < q (long)
      edge_len   [n_edge]    great-circle length of the shared polygon edge
      edge_mid   [n_edge, 3] unit midpoint of that arc
      edge_nrm   [n_edge, 3] unit tangent normal to the arc at its midpoint,
                              pointing from cell p into cell q
      perm_pi2   [n_ang]     index of the direction obtained by a rotation by
                              pi about the 2-axis, (x, y, z) -> (-x, y, -z)
    """

    def __init__(self, N):
        if N < 1:
            raise ValueError("geodesic level must be >= 1")
        self.N = N
        ico, faces = icosahedron()
        points = []          # flat lattice points (not projected)
        index = {}           # dedupe by rounded projected position
        tris = []            # lattice triangles as vertex-index triples
        tri_flat_centroid = []

        def vid(P):
            u = P / np.linalg.norm(P)
            key = tuple(np.round(u * 1e9).astype(np.int64))
            if key not in index:
                index[key] = len(points)
                points.append(P)
            return index[key]

        for (ia, ib, ic) in faces:
            A, B, C = ico[ia], ico[ib], ico[ic]

            def lattice(a, b):
                c = N - a - b
                return (a * A + b * B + c * C) / N

            ids = {}
            for a in range(N + 1):
                for b in range(N + 1 - a):
                    ids[(a, b)] = vid(lattice(a, b))
            for a in range(N + 1):
                for b in range(N + 1 - a):
                    c = N - a - b
                    if c >= 1:      # "up" triangle
                        t = ((a, b), (a + 1, b), (a, b + 1))
                        tris.append(tuple(ids[x] for x in t))
                        tri_flat_centroid.append(sum(lattice(*x) for x in t) / 3.0)
                    if c >= 2:      # "down" triangle
                        t = ((a + 1, b), (a, b + 1), (a + 1, b + 1))
                        tris.append(tuple(ids[x] for x in t))
                        tri_flat_centroid.append(sum(lattice(*x) for x in t) / 3.0)

        n_ang = len(points)
        assert n_ang == 10 * N * N + 2, n_ang
        assert len(tris) == 20 * N * N
        dirs = np.array([p / np.linalg.norm(p) for p in points])
        corners = np.array([c / np.linalg.norm(c) for c in tri_flat_centroid])

        # triangles around every vertex, and the two triangles of every edge
        tri_of_vertex = [[] for _ in range(n_ang)]
        tri_of_edge = {}
        for t, (x, y, z) in enumerate(tris):
            for v in (x, y, z):
                tri_of_vertex[v].append(t)
            for (p, q) in ((x, y), (y, z), (z, x)):
                key = (min(p, q), max(p, q))
                tri_of_edge.setdefault(key, []).append(t)
        assert all(len(ts) == 2 for ts in tri_of_edge.values())
        assert len(tri_of_edge) == 30 * N * N

        # solid angles: order the corners around the centre, fan of triangles
        dOmega = np.zeros(n_ang)
        for v in range(n_ang):
            c = dirs[v]
            e1 = np.cross(c, [0.3, 0.5, 0.7]); e1 /= np.linalg.norm(e1)
            e2 = np.cross(c, e1)
            cs = [corners[t] for t in tri_of_vertex[v]]
            cs.sort(key=lambda x: math.atan2(np.dot(x, e2), np.dot(x, e1)))
            m = len(cs)
            dOmega[v] = sum(_lhuilier(c, cs[k], cs[(k + 1) % m]) for k in range(m))

        edges = sorted(tri_of_edge.keys())
        edge_len, edge_mid, edge_nrm = [], [], []
        nbr = [[] for _ in range(n_ang)]
        for (p, q) in edges:
            t1, t2 = tri_of_edge[(p, q)]
            c1, c2 = corners[t1], corners[t2]
            cr = np.cross(c1, c2)
            edge_len.append(math.atan2(np.linalg.norm(cr), float(np.dot(c1, c2))))
            mid = (c1 + c2) / np.linalg.norm(c1 + c2)
            nu = cr / np.linalg.norm(cr)
            if np.dot(nu, dirs[q] - dirs[p]) < 0.0:
                nu = -nu
            edge_mid.append(mid)
            edge_nrm.append(nu)
            nbr[p].append(q)
            nbr[q].append(p)

        # rotation by pi about the 2-axis (used by the polar boundary)
        rot = dirs * np.array([-1.0, 1.0, -1.0])
        d2 = ((rot[:, None, :] - dirs[None, :, :]) ** 2).sum(-1)
        perm = d2.argmin(axis=1)
        self.perm_err = float(np.sqrt(d2[np.arange(n_ang), perm].max()))

        self.n_ang = n_ang
        self.dir = torch.tensor(dirs, dtype=DTYPE)
        self.dOmega = torch.tensor(dOmega, dtype=DTYPE)
        self.nbr = nbr
        self.edges = torch.tensor(edges, dtype=torch.long)
        self.edge_len = torch.tensor(edge_len, dtype=DTYPE)
        self.edge_mid = torch.tensor(np.array(edge_mid), dtype=DTYPE)
        self.edge_nrm = torch.tensor(np.array(edge_nrm), dtype=DTYPE)
        self.perm_pi2 = torch.tensor(perm, dtype=torch.long)
        self.corners = corners
        self.tri_of_vertex = tri_of_vertex
        self.n_corner = len(tris)


def boost_resolution(dOmega_max, v_max):
    """Smallest N_ang that keeps fluid-frame bins below dOmega_max (end of Sec. 2.6)."""
    return 4.0 * math.pi / dOmega_max * (1.0 + v_max) / (1.0 - v_max)


class LatLongGrid:
    """Latitude-longitude angle grid (Sec. 2.6).

    N_zeta bands bounded by latitude lines equally spaced in cos(zeta) from
    +1 to -1, and N_psi sectors bounded by longitude lines equally spaced in
    psi from 0 to 2 pi: N_zeta N_psi cells of equal solid angle
    4 pi / (N_zeta N_psi).  Readings (the paper states the grid only):
      * the direction of a cell is the point halfway between its bounding
        lines in cos(zeta) and in psi (it splits the cell into equal solid
        angles both ways);
      * the edges are the cell's sides: a meridian arc between two sectors
        (a great-circle arc, length zeta_lo - zeta_hi, midpoint halfway in
        zeta, normal e_psi) and a latitude arc between two bands (a small
        circle, length sin(zeta_b) dpsi, midpoint at the sector's centre,
        normal e_zeta); the polar caps are points and carry no flux;
      * N_psi is even and at least 4, so that the pi rotation about the
        2-axis maps cells to cells and no two cells share two sides.
    Attributes as GeodesicGrid (n_ang, dir, dOmega, nbr, edges, edge_len,
    edge_mid, edge_nrm, perm_pi2), plus
      edge_line  [n_edge, 2]  for the side between p and q: the cell behind p
                              and the cell beyond q on the line through p and
                              q (a band for a meridian side; a sector for a
                              latitude side, continued across a pole into
                              the sector psi + pi of the same band), for
                              reconstruction along the line (Sec. 2.6 reads
                              "the same algorithms as spatial
                              reconstruction": PLM across the poles).
    """

    def __init__(self, n_zeta, n_psi):
        if n_zeta < 1 or n_psi < 4 or n_psi % 2:
            raise ValueError("lat/long grid needs N_zeta >= 1 and an even N_psi >= 4")
        self.n_zeta, self.n_psi = n_zeta, n_psi
        self.n_ang = n_zeta * n_psi
        dpsi = 2.0 * math.pi / n_psi
        cb = [1.0 - 2.0 * i / n_zeta for i in range(n_zeta + 1)]      # cos(zeta) of the latitude lines
        zb = [math.acos(min(1.0, max(-1.0, c))) for c in cb]
        cell = lambda i, j: i * n_psi + (j % n_psi)

        def zeta_line(i, j):
            """Cell i of the line of sector j through both poles (i may be -1 or n_zeta)."""
            if i < 0:
                return cell(0, j + n_psi // 2)
            if i >= n_zeta:
                return cell(n_zeta - 1, j + n_psi // 2)
            return cell(i, j)
        dirs, dOm = [], []
        for i in range(n_zeta):
            cz = 0.5 * (cb[i] + cb[i + 1])
            sz = math.sqrt(max(0.0, 1.0 - cz * cz))
            for j in range(n_psi):
                p = (j + 0.5) * dpsi
                dirs.append((sz * math.cos(p), sz * math.sin(p), cz))
                dOm.append((cb[i] - cb[i + 1]) * dpsi)
        edges = []                      # (a, b, length, mid, normal from a to b, behind a, beyond b)
        for i in range(n_zeta):
            zm = 0.5 * (zb[i] + zb[i + 1])
            for j in range(n_psi):      # meridian at psi_b between sectors j and j + 1
                pb = (j + 1) * dpsi
                edges.append((cell(i, j), cell(i, j + 1), zb[i + 1] - zb[i],
                               (math.sin(zm) * math.cos(pb), math.sin(zm) * math.sin(pb), math.cos(zm)),
                               (-math.sin(pb), math.cos(pb), 0.0), cell(i, j - 1), cell(i, j + 2)))
        for i in range(n_zeta - 1):     # latitude line between bands i and i + 1
            z = zb[i + 1]
            for j in range(n_psi):
                pc = (j + 0.5) * dpsi
                edges.append((cell(i, j), cell(i + 1, j), math.sin(z) * dpsi,
                              (math.sin(z) * math.cos(pc), math.sin(z) * math.sin(pc), math.cos(z)),
                              (math.cos(z) * math.cos(pc), math.cos(z) * math.sin(pc), -math.sin(z)),
                              zeta_line(i - 1, j), zeta_line(i + 2, j)))
        pq, ln, mid, nrm, line = [], [], [], [], []
        self.nbr = [[] for _ in range(self.n_ang)]
        for a, b, length, m, nu, behind, beyond in edges:
            if a > b:                   # store p < q with the normal from p to q
                a, b, nu = b, a, tuple(-x for x in nu)
                behind, beyond = beyond, behind
            pq.append((a, b))
            line.append((behind, beyond))
            ln.append(length)
            mid.append(m)
            nrm.append(nu)
            self.nbr[a].append(b)
            self.nbr[b].append(a)
        self.dir = torch.tensor(dirs, dtype=DTYPE)
        self.dOmega = torch.tensor(dOm, dtype=DTYPE)
        self.edges = torch.tensor(pq, dtype=torch.long)
        self.edge_len = torch.tensor(ln, dtype=DTYPE)
        self.edge_mid = torch.tensor(mid, dtype=DTYPE)
        self.edge_nrm = torch.tensor(nrm, dtype=DTYPE)
        self.edge_line = torch.tensor(line, dtype=torch.long)
        # (x, y, z) -> (-x, y, -z): zeta -> pi - zeta (band i -> N_zeta - 1 - i),
        # psi -> pi - psi (sector j -> N_psi / 2 - 1 - j)
        self.perm_pi2 = torch.tensor([cell(n_zeta - 1 - i, n_psi // 2 - 1 - j)
                                      for i in range(n_zeta) for j in range(n_psi)], dtype=torch.long)
