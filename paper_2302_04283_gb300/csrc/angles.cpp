// Geodesic angle grid builder (host, FP64), Sec. 2.6.
//
// Construction: the 12 vertices of an icosahedron (one on +3hat, the upper
// ring of five at azimuths 2 pi k / 5, the lower ring offset by pi / 5, so
// that the 2hat axis is a two-fold axis); its 20 faces are found as the
// vertex triples at mutual edge distance.  Each face is cut flat into N^2
// triangles on the barycentric lattice a + b + c = N.  Lattice points are
// identified exactly (no floating tolerance) by their integer weights on
// the icosahedron vertices, so points shared by neighbouring faces merge.
// The radiation directions are the projected lattice points; the cell of a
// point is bounded by great-circle arcs through the projected centroids of
// the lattice triangles around it.  Solid angles are sums of
// Van Oosterom-Strackee triangle areas over the fan from the cell centre.
// The cells are numbered so that cells 2t and 2t + 1 have no direction
// component of opposite sign wherever the grid allows it (pair_by_sign).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <numeric>

#include "rad_internal.h"

namespace rad {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return mul(a, 1.0 / norm(a)); }

// Solid angle of the spherical triangle (a, b, c) of unit vectors
// (Van Oosterom & Strackee 1983).
double vos_area(V3 a, V3 b, V3 c) {
  double num = std::fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * std::atan2(num, den);
}

// Exact identity of a lattice point: sorted (vertex, weight) pairs.
uint64_t lattice_key(std::array<std::pair<int, int>, 3> w) {
  std::sort(w.begin(), w.end());
  uint64_t key = 0;
  for (auto &p : w) {
    if (p.second == 0) continue;
    key = key * 1024u + (uint64_t)(p.first * 64 + p.second);
  }
  return key;
}

// Renumber the lattice points so that points 2t and 2t + 1 have no
// coordinate of opposite sign (a zero coordinate agrees with either sign).
// A thread of the stage kernel owns such a pair of bins, so in flat
// Cartesian space both of its bins take their upwind states from the same
// side of the cell in every dimension.  Greedy matching: the points with
// the most nonzero coordinates first, in order of sign pattern, each taking
// the next unmatched compatible point (one of its own pattern when any is
// left, since those follow it in this order).  Points left without a partner
// are paired in order at the end; returns whether there were none.
bool pair_by_sign(std::vector<V3> &flat, std::vector<std::array<int, 3>> &tris) {
  const int n = (int)flat.size();
  std::vector<std::array<int, 3>> sg(n);
  std::vector<int> nnz(n, 0);
  for (int a = 0; a < n; ++a) {
    const double c[3] = {flat[a].x, flat[a].y, flat[a].z};
    const double tol = 1e-12 * norm(flat[a]);
    for (int k = 0; k < 3; ++k) {
      sg[a][k] = c[k] > tol ? 1 : (c[k] < -tol ? -1 : 0);
      nnz[a] += sg[a][k] != 0;
    }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (nnz[a] != nnz[b]) return nnz[a] > nnz[b];
    return sg[a] < sg[b];
  });
  auto compatible = [&](int a, int b) {
    for (int k = 0; k < 3; ++k)
      if (sg[a][k] * sg[b][k] < 0) return false;
    return true;
  };
  std::vector<char> used(n, 0);
  std::vector<int> seq, rest;
  seq.reserve(n);
  for (int ia = 0; ia < n; ++ia) {
    const int a = order[ia];
    if (used[a]) continue;
    used[a] = 1;
    int pick = -1;
    for (int ib = ia + 1; ib < n && pick < 0; ++ib)
      if (!used[order[ib]] && compatible(a, order[ib])) pick = order[ib];
    if (pick < 0) {
      rest.push_back(a);
      continue;
    }
    used[pick] = 1;
    seq.push_back(a);
    seq.push_back(pick);
  }
  const bool all = rest.empty();
  seq.insert(seq.end(), rest.begin(), rest.end());
  std::vector<int> newid(n);
  std::vector<V3> f2(n);
  for (int i = 0; i < n; ++i) {
    newid[seq[i]] = i;
    f2[i] = flat[seq[i]];
  }
  flat.swap(f2);
  for (auto &t : tris)
    for (int k = 0; k < 3; ++k) t[k] = newid[t[k]];
  return all;
}

// Bin of the direction rotated by pi about 2hat, (x, y, z) -> (-x, y, -z),
// by nearest direction; fails unless the grid is symmetric under it.
bool pi_rotation_perm(AngleGrid &g, std::string &err) {
  const int n_ang = g.n_ang;
  g.perm.assign(n_ang, -1);
  for (int n = 0; n < n_ang; ++n) {
    const double rx = -g.dir[3 * n], ry = g.dir[3 * n + 1], rz = -g.dir[3 * n + 2];
    int best = -1;
    double bd = 1e9;
    for (int m = 0; m < n_ang; ++m) {
      const double dx = rx - g.dir[3 * m], dy = ry - g.dir[3 * m + 1], dz = rz - g.dir[3 * m + 2];
      const double dd = dx * dx + dy * dy + dz * dz;
      if (dd < bd) {
        bd = dd;
        best = m;
      }
    }
    if (bd > 1e-24) {
      err = "angle grid is not symmetric under the pi rotation about 2hat";
      return false;
    }
    g.perm[n] = best;
  }
  return true;
}

}  // namespace

// Minimum-angle plane reconstruction on a geodesic grid: per cell its
// neighbours in cyclic order around n, for each two cyclically adjacent ones
// (a, b) the inverse of [x_a; x_b] (gnomonic coordinates x = (v . t1,
// v . t2) / (v . n) in the tangent plane at n, any orthonormal t1, t2), so
// that the plane's gradient is g = inv (I_a - I_c, I_b - I_c); and per slot
// the gnomonic coordinates of the side's midpoint in this cell's and in the
// neighbour's tangent plane.
static void build_mapr(AngleGrid &g, const std::vector<V3> &dir) {
  const int n_ang = g.n_ang;
  std::vector<V3> t1(n_ang), t2(n_ang);
  for (int c = 0; c < n_ang; ++c) {
    const V3 n = dir[c];
    const V3 a = std::fabs(n.z) < 0.9 ? V3{0.0, 0.0, 1.0} : V3{1.0, 0.0, 0.0};
    t1[c] = unit(cross(n, a));
    t2[c] = cross(n, t1[c]);
  }
  auto gn = [&](int c, V3 v, double &x, double &y) {
    const double w = dot(v, dir[c]);
    x = dot(v, t1[c]) / w;
    y = dot(v, t2[c]) / w;
  };
  g.mapr_nb.assign(6 * n_ang, -1);
  g.mapr_minv.assign(24 * n_ang, 0.0);
  g.mapr_xo.assign(12 * n_ang, 0.0);
  g.mapr_xn.assign(12 * n_ang, 0.0);
  for (int c = 0; c < n_ang; ++c) {
    std::vector<std::pair<double, int>> cyc;
    for (int s = 0; s < 6; ++s) {
      const int m = g.nbr[6 * c + s];
      if (m < 0) continue;
      double x, y;
      gn(c, dir[m], x, y);
      cyc.push_back({std::atan2(y, x), m});
    }
    std::sort(cyc.begin(), cyc.end());
    const int K = (int)cyc.size();
    for (int a = 0; a < K; ++a) g.mapr_nb[6 * c + a] = cyc[a].second;
    for (int a = 0; a < K; ++a) {
      double xa, ya, xb, yb;
      gn(c, dir[cyc[a].second], xa, ya);
      gn(c, dir[cyc[(a + 1) % K].second], xb, yb);
      const double det = xa * yb - ya * xb;           // rows (xa, ya), (xb, yb)
      double *mi = &g.mapr_minv[24 * c + 4 * a];
      mi[0] = yb / det;
      mi[1] = -ya / det;
      mi[2] = -xb / det;
      mi[3] = xa / det;
    }
    for (int s = 0; s < 6; ++s) {
      const int m = g.nbr[6 * c + s];
      if (m < 0) continue;
      const int e = g.slot_edge[6 * c + s];
      const V3 mid{g.edge_mid[3 * e], g.edge_mid[3 * e + 1], g.edge_mid[3 * e + 2]};
      gn(c, mid, g.mapr_xo[12 * c + 2 * s], g.mapr_xo[12 * c + 2 * s + 1]);
      gn(m, mid, g.mapr_xn[12 * c + 2 * s], g.mapr_xn[12 * c + 2 * s + 1]);
    }
  }
}

bool build_geodesic(int N, AngleGrid &g, std::string &err) {
  if (N < 1 || N > 32) {
    err = "geodesic level must be in [1, 32]";
    return false;
  }
  // icosahedron
  std::vector<V3> ico;
  const double h = 1.0 / std::sqrt(5.0), r = 2.0 / std::sqrt(5.0);
  ico.push_back({0.0, 0.0, 1.0});
  for (int k = 0; k < 5; ++k) {
    double psi = 2.0 * kPi * k / 5.0;
    ico.push_back({r * std::cos(psi), r * std::sin(psi), h});
  }
  for (int k = 0; k < 5; ++k) {
    double psi = 2.0 * kPi * k / 5.0 + kPi / 5.0;
    ico.push_back({r * std::cos(psi), r * std::sin(psi), -h});
  }
  ico.push_back({0.0, 0.0, -1.0});
  double edge2 = 1e9;
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b) edge2 = std::min(edge2, dot(sub(ico[a], ico[b]), sub(ico[a], ico[b])));
  auto adjacent = [&](int a, int b) {
    V3 d = sub(ico[a], ico[b]);
    return std::fabs(dot(d, d) - edge2) < 1e-9;
  };
  std::vector<std::array<int, 3>> faces;
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b)
      for (int c = b + 1; c < 12; ++c)
        if (adjacent(a, b) && adjacent(b, c) && adjacent(a, c)) faces.push_back({a, b, c});
  if (faces.size() != 20) {
    err = "icosahedron face search failed";
    return false;
  }

  std::map<uint64_t, int> ids;
  std::vector<V3> flat;                   // unprojected lattice points
  std::vector<std::array<int, 3>> tris;   // lattice triangles
  std::vector<V3> tri_centroid;           // projected centroids (polygon corners)
  for (auto &f : faces) {
    auto point = [&](int a, int b) {
      int c = N - a - b;
      V3 p = add(add(mul(ico[f[0]], a), mul(ico[f[1]], b)), mul(ico[f[2]], c));
      return mul(p, 1.0 / N);
    };
    auto id = [&](int a, int b) {
      int c = N - a - b;
      uint64_t key = lattice_key({std::make_pair(f[0], a), std::make_pair(f[1], b), std::make_pair(f[2], c)});
      auto it = ids.find(key);
      if (it != ids.end()) return it->second;
      int n = (int)flat.size();
      ids[key] = n;
      flat.push_back(point(a, b));
      return n;
    };
    for (int a = 0; a <= N; ++a)
      for (int b = 0; a + b <= N; ++b) {
        int c = N - a - b;
        if (c >= 1) {
          tris.push_back({id(a, b), id(a + 1, b), id(a, b + 1)});
          tri_centroid.push_back(unit(add(add(point(a, b), point(a + 1, b)), point(a, b + 1))));
        }
        if (c >= 2) {
          tris.push_back({id(a + 1, b), id(a, b + 1), id(a + 1, b + 1)});
          tri_centroid.push_back(unit(add(add(point(a + 1, b), point(a, b + 1)), point(a + 1, b + 1))));
        }
      }
  }
  const int n_ang = (int)flat.size();
  if (n_ang != 10 * N * N + 2 || (int)tris.size() != 20 * N * N) {
    err = "geodesic grid has the wrong cell count";
    return false;
  }
  const bool paired = pair_by_sign(flat, tris);
  std::vector<V3> dir(n_ang);
  for (int n = 0; n < n_ang; ++n) dir[n] = unit(flat[n]);

  // triangles around vertices and the two triangles of each lattice edge
  std::vector<std::vector<int>> vtris(n_ang);
  std::map<std::pair<int, int>, std::vector<int>> etris;
  for (int t = 0; t < (int)tris.size(); ++t) {
    for (int k = 0; k < 3; ++k) {
      vtris[tris[t][k]].push_back(t);
      int p = tris[t][k], q = tris[t][(k + 1) % 3];
      etris[{std::min(p, q), std::max(p, q)}].push_back(t);
    }
  }
  if ((int)etris.size() != 30 * N * N) {
    err = "geodesic grid has the wrong edge count";
    return false;
  }

  g = AngleGrid();
  g.level = N;
  g.n_ang = n_ang;
  g.sign_pairs = paired;
  g.n_ap = (n_ang + 3) / 4 * 4;
  g.dir.resize(3 * n_ang);
  g.dOmega.resize(n_ang);
  for (int n = 0; n < n_ang; ++n) {
    g.dir[3 * n] = dir[n].x;
    g.dir[3 * n + 1] = dir[n].y;
    g.dir[3 * n + 2] = dir[n].z;
    // order the corners by angle in the tangent plane, then sum the fan
    V3 c = dir[n];
    V3 t1 = unit(cross(c, V3{0.3, 0.5, 0.7}));
    V3 t2 = cross(c, t1);
    std::vector<std::pair<double, V3>> cs;
    for (int t : vtris[n]) {
      V3 p = tri_centroid[t];
      cs.push_back({std::atan2(dot(p, t2), dot(p, t1)), p});
    }
    std::sort(cs.begin(), cs.end(), [](const std::pair<double, V3> &a, const std::pair<double, V3> &b) {
      return a.first < b.first;
    });
    double area = 0.0;
    for (size_t k = 0; k < cs.size(); ++k) area += vos_area(c, cs[k].second, cs[(k + 1) % cs.size()].second);
    g.dOmega[n] = area;
  }

  g.n_edge = (int)etris.size();
  g.nbr.assign(6 * n_ang, -1);
  g.slot_edge.assign(6 * n_ang, -1);
  std::vector<std::vector<std::pair<int, int>>> nb(n_ang);
  int e = 0;
  for (auto &kv : etris) {
    int p = kv.first.first, q = kv.first.second;
    V3 c1 = tri_centroid[kv.second[0]], c2 = tri_centroid[kv.second[1]];
    V3 cr = cross(c1, c2);
    double len = std::atan2(norm(cr), dot(c1, c2));
    V3 mid = unit(add(c1, c2));
    V3 nu = unit(cr);
    if (dot(nu, sub(dir[q], dir[p])) < 0.0) nu = mul(nu, -1.0);
    g.edge_pq.push_back(p);
    g.edge_pq.push_back(q);
    g.edge_mid.insert(g.edge_mid.end(), {mid.x, mid.y, mid.z});
    g.edge_nrm.insert(g.edge_nrm.end(), {nu.x, nu.y, nu.z});
    g.edge_len.push_back(len);
    nb[p].push_back({q, e});
    nb[q].push_back({p, e});
    ++e;
  }
  for (int n = 0; n < n_ang; ++n) {
    std::sort(nb[n].begin(), nb[n].end());
    if (nb[n].size() < 5 || nb[n].size() > 6) {
      err = "geodesic cell with an unexpected number of neighbours";
      return false;
    }
    for (size_t s = 0; s < nb[n].size(); ++s) {
      g.nbr[6 * n + s] = nb[n][s].first;
      g.slot_edge[6 * n + s] = nb[n][s].second;
    }
  }
  build_mapr(g, dir);
  return pi_rotation_perm(g, err);
}

// Latitude-longitude grid (Sec. 2.6): n_zeta bands between latitude lines
// equally spaced in cos(zeta) from +1 to -1, n_psi sectors between
// longitude lines equally spaced in psi from 0 to 2 pi, every cell of solid
// angle 4 pi / (n_zeta n_psi).  A cell's direction lies halfway between its
// lines in cos(zeta) and in psi.  Its sides: meridian arcs to the
// neighbouring sectors (great circles: length = the zeta extent, midpoint
// halfway in zeta, normal e_psi) and latitude arcs to the neighbouring
// bands (small circles: length sin(zeta) dpsi, midpoint at the sector's
// centre, normal e_zeta); the poles are points and carry no flux.  Cell
// index n = band * n_psi + sector.
bool build_latlong(int n_zeta, int n_psi, AngleGrid &g, std::string &err) {
  if (n_zeta < 1 || n_psi < 4 || (n_psi & 1) || (long long)n_zeta * n_psi > 4096) {
    err = "lat/long grid needs n_zeta >= 1, an even n_psi >= 4 and at most 4096 cells";
    return false;
  }
  g = AngleGrid();
  g.level = 0;
  g.n_ang = n_zeta * n_psi;
  g.n_ap = (g.n_ang + 3) / 4 * 4;
  const double dpsi = 2.0 * kPi / n_psi;
  std::vector<double> cz(n_zeta + 1), zl(n_zeta + 1);
  for (int i = 0; i <= n_zeta; ++i) {
    cz[i] = 1.0 - 2.0 * i / n_zeta;
    zl[i] = std::acos(std::min(1.0, std::max(-1.0, cz[i])));
  }
  g.dir.resize(3 * g.n_ang);
  g.dOmega.resize(g.n_ang);
  for (int i = 0; i < n_zeta; ++i) {
    const double c = 0.5 * (cz[i] + cz[i + 1]), sn = std::sqrt(std::max(0.0, 1.0 - c * c));
    for (int j = 0; j < n_psi; ++j) {
      const int n = i * n_psi + j;
      const double p = (j + 0.5) * dpsi;
      g.dir[3 * n] = sn * std::cos(p);
      g.dir[3 * n + 1] = sn * std::sin(p);
      g.dir[3 * n + 2] = c;
      g.dOmega[n] = (cz[i] - cz[i + 1]) * dpsi;
    }
  }
  std::vector<std::vector<std::pair<int, int>>> nb(g.n_ang);
  // the cell at band i of the line of sector j through both poles (i = -1
  // or n_zeta continues across the pole into sector j + n_psi / 2)
  auto zeta_line = [&](int i, int j) {
    if (i < 0) return (j + n_psi / 2) % n_psi;
    if (i >= n_zeta) return (n_zeta - 1) * n_psi + (j + n_psi / 2) % n_psi;
    return i * n_psi + j;
  };
  // side between cells a and b; behind = the cell before a, beyond = the cell
  // after b on the line through them (for reconstruction along the line)
  auto add_edge = [&](int a, int b, double len, V3 mid, V3 nu, int behind, int beyond) {
    if (a > b) {
      std::swap(a, b);
      std::swap(behind, beyond);
      nu = mul(nu, -1.0);
    }
    const int e = g.n_edge++;
    g.edge_pq.push_back(a);
    g.edge_pq.push_back(b);
    g.edge_line.push_back(behind);
    g.edge_line.push_back(beyond);
    g.edge_mid.insert(g.edge_mid.end(), {mid.x, mid.y, mid.z});
    g.edge_nrm.insert(g.edge_nrm.end(), {nu.x, nu.y, nu.z});
    g.edge_len.push_back(len);
    nb[a].push_back({b, e});
    nb[b].push_back({a, e});
  };
  for (int i = 0; i < n_zeta; ++i) {
    const double zm = 0.5 * (zl[i] + zl[i + 1]);
    for (int j = 0; j < n_psi; ++j) {            // meridian between sectors j and j + 1
      const double pb = (j + 1) * dpsi;
      add_edge(i * n_psi + j, i * n_psi + (j + 1) % n_psi, zl[i + 1] - zl[i],
               V3{std::sin(zm) * std::cos(pb), std::sin(zm) * std::sin(pb), std::cos(zm)},
               V3{-std::sin(pb), std::cos(pb), 0.0}, i * n_psi + (j + n_psi - 1) % n_psi,
               i * n_psi + (j + 2) % n_psi);
    }
  }
  for (int i = 0; i + 1 < n_zeta; ++i) {
    const double z = zl[i + 1];
    for (int j = 0; j < n_psi; ++j) {            // latitude line between bands i and i + 1
      const double pc = (j + 0.5) * dpsi;
      add_edge(i * n_psi + j, (i + 1) * n_psi + j, std::sin(z) * dpsi,
               V3{std::sin(z) * std::cos(pc), std::sin(z) * std::sin(pc), std::cos(z)},
               V3{std::cos(z) * std::cos(pc), std::cos(z) * std::sin(pc), -std::sin(z)}, zeta_line(i - 1, j),
               zeta_line(i + 2, j));
    }
  }
  g.nbr.assign(6 * g.n_ang, -1);
  g.slot_edge.assign(6 * g.n_ang, -1);
  for (int n = 0; n < g.n_ang; ++n) {
    std::sort(nb[n].begin(), nb[n].end());
    if (nb[n].size() > 6) {
      err = "lat/long cell with more than six sides";
      return false;
    }
    for (size_t s = 0; s < nb[n].size(); ++s) {
      g.nbr[6 * n + s] = nb[n][s].first;
      g.slot_edge[6 * n + s] = nb[n][s].second;
    }
  }
  // the inverse of edge_line: per bin, the sides whose line reconstruction
  // (from p, or from q) takes it as the cell behind
  g.line_behind.assign(kMaxBehind * g.n_ang, -1);
  std::vector<int> cnt(g.n_ang, 0);
  for (int e = 0; e < g.n_edge; ++e)
    for (int s = 0; s < 2; ++s) {
      const int t = g.edge_line[2 * e + s];
      if (cnt[t] == kMaxBehind) {
        err = "lat/long cell behind more than four sides";
        return false;
      }
      g.line_behind[kMaxBehind * t + cnt[t]++] = 2 * e + s;
    }
  return pi_rotation_perm(g, err);
}

}  // namespace rad
