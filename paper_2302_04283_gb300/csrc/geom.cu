// Geometry precompute (FP64), Secs. 2.1-2.2.
//
// One thread per (i, j) column evaluates, at the cell centre, the metric,
// the normal-observer tetrad (Eq. tetrad; spatial legs by Gram-Schmidt with
// the spatial metric), M = g e, the Ricci rotation coefficients (Eq. ricci)
// and the exact cell volume; other threads evaluate face tetrad rows and
// exact face areas.  Coordinate derivatives come from forward-mode dual
// numbers carrying d/dx1, d/dx2, d/dx3 through the analytic metric, so the
// rotation coefficients are exact to rounding.  The metrics are stationary
// and independent of x3, so one column serves every k.
#include <cmath>
#include <cstring>

#include "rad_internal.h"

namespace rad {
namespace {

struct Dual {
  double v, d[3];
};
__device__ __forceinline__ Dual dconst(double v) { return {v, {0.0, 0.0, 0.0}}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) {
  return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
__device__ __forceinline__ Dual operator-(Dual a, Dual b) {
  return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, {-a.d[0], -a.d[1], -a.d[2]}}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) {
  return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2]}}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  double iv = 1.0 / b.v;
  double q = a.v * iv;
  return {q, {(a.d[0] - q * b.d[0]) * iv, (a.d[1] - q * b.d[1]) * iv, (a.d[2] - q * b.d[2]) * iv}};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
  double s = sqrt(a.v);
  double h = 0.5 / s;
  return {s, {a.d[0] * h, a.d[1] * h, a.d[2] * h}};
}
__device__ __forceinline__ Dual dsin(Dual a) {
  double s = sin(a.v), c = cos(a.v);
  return {s, {c * a.d[0], c * a.d[1], c * a.d[2]}};
}
__device__ __forceinline__ Dual dcos(Dual a) {
  double s = sin(a.v), c = cos(a.v);
  return {c, {-s * a.d[0], -s * a.d[1], -s * a.d[2]}};
}

// g_{mu nu}(x) for the three spacetimes.
__device__ void metric(int kind, double a, const Dual x[3], Dual g[4][4]) {
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) g[m][n] = dconst(0.0);
  if (kind == RAD_MINK_CART) {
    g[0][0] = dconst(-1.0);
    g[1][1] = g[2][2] = g[3][3] = dconst(1.0);
  } else if (kind == RAD_MINK_SPH) {
    Dual r = x[0], s = dsin(x[1]);
    g[0][0] = dconst(-1.0);
    g[1][1] = dconst(1.0);
    g[2][2] = r * r;
    g[3][3] = r * r * s * s;
  } else {  // Kerr-Schild, M = 1
    Dual r = x[0], s = dsin(x[1]), c = dcos(x[1]);
    Dual sig = r * r + (a * a) * (c * c);
    Dual q = 2.0 * r / sig;
    Dual s2 = s * s;
    g[0][0] = q - dconst(1.0);
    g[0][1] = g[1][0] = q;
    g[0][3] = g[3][0] = -a * (q * s2);
    g[1][1] = dconst(1.0) + q;
    g[1][3] = g[3][1] = -a * ((dconst(1.0) + q) * s2);
    g[2][2] = sig;
    g[3][3] = s2 * (r * r + dconst(a * a) + (a * a) * (q * s2));
  }
}

// e[mu][A] = e^mu_A with e_0 the normal observer and the spatial legs
// Gram-Schmidt'ed in the metric's order.
__device__ void tetrad(int kind, const Dual g[4][4], Dual e[4][4]) {
  // spatial metric inverse by cofactors
  Dual gm[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) gm[a][b] = g[a + 1][b + 1];
  Dual c00 = gm[1][1] * gm[2][2] - gm[1][2] * gm[2][1];
  Dual c01 = gm[1][2] * gm[2][0] - gm[1][0] * gm[2][2];
  Dual c02 = gm[1][0] * gm[2][1] - gm[1][1] * gm[2][0];
  Dual det = gm[0][0] * c00 + gm[0][1] * c01 + gm[0][2] * c02;
  Dual inv[3][3];
  inv[0][0] = c00 / det;
  inv[1][0] = c01 / det;
  inv[2][0] = c02 / det;
  inv[0][1] = (gm[0][2] * gm[2][1] - gm[0][1] * gm[2][2]) / det;
  inv[1][1] = (gm[0][0] * gm[2][2] - gm[0][2] * gm[2][0]) / det;
  inv[2][1] = (gm[0][1] * gm[2][0] - gm[0][0] * gm[2][1]) / det;
  inv[0][2] = (gm[0][1] * gm[1][2] - gm[0][2] * gm[1][1]) / det;
  inv[1][2] = (gm[0][2] * gm[1][0] - gm[0][0] * gm[1][2]) / det;
  inv[2][2] = (gm[0][0] * gm[1][1] - gm[0][1] * gm[1][0]) / det;
  // shift beta^a = gamma^{ab} g_{0b}, lapse^2 = beta^a g_{0a} - g_00
  Dual beta[3];
  Dual lap2 = -g[0][0];
  for (int a = 0; a < 3; ++a) {
    beta[a] = inv[a][0] * g[0][1] + inv[a][1] * g[0][2] + inv[a][2] * g[0][3];
    lap2 = lap2 + beta[a] * g[0][a + 1];
  }
  Dual lap = dsqrt(lap2);
  for (int m = 0; m < 4; ++m)
    for (int A = 0; A < 4; ++A) e[m][A] = dconst(0.0);
  e[0][0] = dconst(1.0) / lap;
  for (int a = 0; a < 3; ++a) e[a + 1][0] = -beta[a] / lap;
  int coord[3], leg[3];
  if (kind == RAD_MINK_CART) {
    coord[0] = 2; leg[0] = 3;    // z -> 3hat
    coord[1] = 0; leg[1] = 1;    // x -> 1hat
    coord[2] = 1; leg[2] = 2;    // y -> 2hat
  } else {
    coord[0] = 1; leg[0] = 3;    // theta -> 3hat
    coord[1] = 2; leg[1] = 1;    // phi -> 1hat
    coord[2] = 0; leg[2] = 2;    // r -> 2hat
  }
  Dual basis[3][3];
  for (int s = 0; s < 3; ++s) {
    Dual v[3];
    for (int a = 0; a < 3; ++a) v[a] = dconst(a == coord[s] ? 1.0 : 0.0);
    for (int t = 0; t < s; ++t) {
      Dual pr = dconst(0.0);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) pr = pr + basis[t][a] * gm[a][b] * v[b];
      for (int a = 0; a < 3; ++a) v[a] = v[a] - pr * basis[t][a];
    }
    Dual nn = dconst(0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) nn = nn + v[a] * gm[a][b] * v[b];
    Dual inv_n = dconst(1.0) / dsqrt(nn);
    for (int a = 0; a < 3; ++a) {
      basis[s][a] = v[a] * inv_n;
      e[a + 1][leg[s]] = basis[s][a];
    }
  }
}

__device__ double cell_volume(int kind, double a, const double lo[3], const double hi[3]) {
  if (kind == RAD_MINK_CART) return (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  double aa = (kind == RAD_KS_SPH) ? a * a : 0.0;
  double c1 = cos(lo[1]), c2 = cos(hi[1]);
  return (hi[2] - lo[2]) * ((hi[0] * hi[0] * hi[0] - lo[0] * lo[0] * lo[0]) / 3.0 * (c1 - c2) +
                            aa * (hi[0] - lo[0]) * (c1 * c1 * c1 - c2 * c2 * c2) / 3.0);
}

// Exact area of the face at x_d = lo[d]; lo/hi give the other extents.
__device__ double face_area(int kind, double a, int d, const double lo[3], const double hi[3]) {
  if (kind == RAD_MINK_CART) {
    double w[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    return d == 0 ? w[1] * w[2] : (d == 1 ? w[0] * w[2] : w[0] * w[1]);
  }
  double aa = (kind == RAD_KS_SPH) ? a * a : 0.0;
  double c1 = cos(lo[1]), c2 = cos(hi[1]);
  if (d == 0) return (hi[2] - lo[2]) * (lo[0] * lo[0] * (c1 - c2) + aa * (c1 * c1 * c1 - c2 * c2 * c2) / 3.0);
  if (d == 1)
    return (hi[2] - lo[2]) * sin(lo[1]) *
           ((hi[0] * hi[0] * hi[0] - lo[0] * lo[0] * lo[0]) / 3.0 + aa * c1 * c1 * (hi[0] - lo[0]));
  return (hi[0] * hi[0] * hi[0] - lo[0] * lo[0] * lo[0]) / 3.0 * (c1 - c2) +
         aa * (hi[0] - lo[0]) * (c1 * c1 * c1 - c2 * c2 * c2) / 3.0;
}

struct GeomArgs {
  int kind;
  double spin;
  int n1, n2, n3;
  const double *xf1, *xf2, *xf3;
  int polar_lo, polar_hi;  // x2 faces 0 / n2 lie on the polar axis
  ColGeo *cols;
  FaceGeo *f1, *f2, *f3;
};

__global__ void k_geom_cols(GeomArgs A) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n1 * A.n2) return;
  int i = c % A.n1, j = c / A.n1;
  double x1 = 0.5 * (A.xf1[i] + A.xf1[i + 1]);
  double x2 = 0.5 * (A.xf2[j] + A.xf2[j + 1]);
  double x3 = 0.5 * (A.xf3[0] + A.xf3[1]);
  Dual x[3] = {{x1, {1.0, 0.0, 0.0}}, {x2, {0.0, 1.0, 0.0}}, {x3, {0.0, 0.0, 1.0}}};
  Dual g[4][4], e[4][4];
  metric(A.kind, A.spin, x, g);
  tetrad(A.kind, g, e);
  ColGeo out;
  out.n0up = e[0][0].v;
  for (int m = 0; m < 4; ++m)
    for (int B = 0; B < 4; ++B) {
      out.e[m][B] = e[m][B].v;
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += g[m][v].v * e[v][B].v;
      out.M[m][B] = s;
    }
  // Christoffel symbols of the first kind, Gamma_{s d r} = 1/2 (d_d g_sr + d_r g_sd - d_s g_dr)
  auto dg = [&](int m, int n, int d) { return d == 0 ? 0.0 : g[m][n].d[d - 1]; };
  double Gam[4][4][4];
  for (int s = 0; s < 4; ++s)
    for (int d = 0; d < 4; ++d)
      for (int r = 0; r < 4; ++r) Gam[s][d][r] = 0.5 * (dg(s, r, d) + dg(s, d, r) - dg(d, r, s));
  // omega_{C A B} = e^s_C e^d_B (g_{es} d_d e^e_A + Gamma_{s d r} e^r_A), C lowered with eta
  double om[4][4][4];
  for (int C = 0; C < 4; ++C)
    for (int Aa = 0; Aa < 4; ++Aa)
      for (int B = 0; B < 4; ++B) {
        double acc = 0.0;
        for (int s = 0; s < 4; ++s) {
          double esC = e[s][C].v;
          if (esC == 0.0) continue;
          for (int d = 0; d < 4; ++d) {
            double edB = e[d][B].v;
            if (edB == 0.0) continue;
            double t = 0.0;
            for (int ee = 0; ee < 4; ++ee) t += g[ee][s].v * (d == 0 ? 0.0 : e[ee][Aa].d[d - 1]);
            for (int r = 0; r < 4; ++r) t += Gam[s][d][r] * e[r][Aa].v;
            acc += esC * edB * t;
          }
        }
        om[C][Aa][B] = (C == 0) ? -acc : acc;   // raise C with eta
      }
  const int pa[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
  const int pb[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
  for (int ii = 0; ii < 3; ++ii)
    for (int p = 0; p < 10; ++p) {
      int a0 = pa[p], b0 = pb[p];
      out.K[ii][p] = (a0 == b0) ? om[ii + 1][a0][b0] : om[ii + 1][a0][b0] + om[ii + 1][b0][a0];
    }
  for (int p = 0; p < 10; ++p) {
    int a0 = pa[p], b0 = pb[p];
    out.K0[p] = (a0 == b0) ? om[0][a0][b0] : om[0][a0][b0] + om[0][b0][a0];
  }
  double lo[3] = {A.xf1[i], A.xf2[j], A.xf3[0]}, hi[3] = {A.xf1[i + 1], A.xf2[j + 1], A.xf3[1]};
  out.dV = cell_volume(A.kind, A.spin, lo, hi);
  out.invdV = 1.0 / out.dV;
  A.cols[c] = out;
  // x3 faces (uniform along x3): the cell-centre tetrad, area over (x1, x2)
  FaceGeo f;
  for (int B = 0; B < 4; ++B) {
    f.ea[B] = out.e[3][B];
    f.m0[B] = out.M[0][B];
  }
  f.dA = face_area(A.kind, A.spin, 2, lo, hi);
  f.pad[0] = f.pad[1] = f.pad[2] = 0.0;
  A.f3[c] = f;
}

// d = 0: faces [n2][n1+1] at (xf1[i], x2c[j]); d = 1: faces [n2+1][n1] at (x1c[i], xf2[j]).
__global__ void k_geom_faces(GeomArgs A, int d) {
  int nf1 = (d == 0) ? A.n1 + 1 : A.n1;
  int nf2 = (d == 1) ? A.n2 + 1 : A.n2;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nf1 * nf2) return;
  int i = c % nf1, j = c / nf1;
  FaceGeo f;
  for (int B = 0; B < 4; ++B) f.ea[B] = f.m0[B] = 0.0;
  f.pad[0] = f.pad[1] = f.pad[2] = 0.0;
  bool polar = (d == 1) && ((j == 0 && A.polar_lo) || (j == A.n2 && A.polar_hi));
  if (polar) {
    f.dA = 0.0;   // the polar axis has zero area: no flux crosses it
  } else {
    double x1 = (d == 0) ? A.xf1[i] : 0.5 * (A.xf1[i] + A.xf1[i + 1]);
    double x2 = (d == 1) ? A.xf2[j] : 0.5 * (A.xf2[j] + A.xf2[j + 1]);
    double x3 = 0.5 * (A.xf3[0] + A.xf3[1]);
    Dual x[3] = {dconst(x1), dconst(x2), dconst(x3)};
    Dual g[4][4], e[4][4];
    metric(A.kind, A.spin, x, g);
    tetrad(A.kind, g, e);
    for (int B = 0; B < 4; ++B) {
      f.ea[B] = e[d + 1][B].v;
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += g[0][v].v * e[v][B].v;
      f.m0[B] = s;
    }
    double lo[3], hi[3];
    if (d == 0) {
      lo[0] = A.xf1[i]; hi[0] = A.xf1[i];
      lo[1] = A.xf2[j]; hi[1] = A.xf2[j + 1];
    } else {
      lo[0] = A.xf1[i]; hi[0] = A.xf1[i + 1];
      lo[1] = A.xf2[j]; hi[1] = A.xf2[j];
    }
    lo[2] = A.xf3[0];
    hi[2] = A.xf3[1];
    f.dA = face_area(A.kind, A.spin, d, lo, hi);
  }
  (d == 0 ? A.f1 : A.f2)[c] = f;
}

__global__ void k_cols_to_f32(const ColGeo *in, ColGeoF *out, int n) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const ColGeo &a = in[c];
  ColGeoF b;
  b.n0up = (float)a.n0up;
  b.invdV = (float)a.invdV;
  b.dV = (float)a.dV;
  b.pad = 0.0f;
  for (int m = 0; m < 4; ++m)
    for (int B = 0; B < 4; ++B) {
      b.M[m][B] = (float)a.M[m][B];
      b.e[m][B] = (float)a.e[m][B];
    }
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < 10; ++p) b.K[i][p] = (float)a.K[i][p];
  b.pad2[0] = b.pad2[1] = 0.0f;
  for (int p = 0; p < 10; ++p) b.K0[p] = (float)a.K0[p];
  b.pad3[0] = b.pad3[1] = 0.0f;
  out[c] = b;
}

__global__ void k_faces_to_f32(const FaceGeo *in, FaceGeoF *out, int n) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const FaceGeo &a = in[c];
  FaceGeoF b;
  for (int B = 0; B < 4; ++B) {
    b.ea[B] = (float)a.ea[B];
    b.m0[B] = (float)a.m0[B];
  }
  b.dA = (float)a.dA;
  b.pad[0] = b.pad[1] = b.pad[2] = 0.0f;
  out[c] = b;
}

}  // namespace

void free_geometry(DevGeom &g) {
  cudaFree(g.cols);
  cudaFree(g.f1);
  cudaFree(g.f2);
  cudaFree(g.f3);
  cudaFree(g.colsF);
  cudaFree(g.f1F);
  cudaFree(g.f2F);
  cudaFree(g.f3F);
  cudaFree(g.xf_dev);
  g.cols = nullptr;
  g.f1 = g.f2 = g.f3 = nullptr;
  g.colsF = nullptr;
  g.f1F = g.f2F = g.f3F = nullptr;
  g.xf_dev = nullptr;
}

int compute_geometry(rad_ctx *ctx, std::string &err) {
  DevGeom &G = ctx->geom;
  free_geometry(G);
  const int n1 = G.n[0], n2 = G.n[1], n3 = G.n[2];
  size_t ncol = (size_t)n1 * n2;
  size_t nx = G.xf[0].size() + G.xf[1].size() + 2;
  cudaError_t ce;
  if ((ce = cudaMalloc(&G.cols, ncol * sizeof(ColGeo))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f1, (size_t)n2 * (n1 + 1) * sizeof(FaceGeo))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f2, (size_t)(n2 + 1) * n1 * sizeof(FaceGeo))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f3, ncol * sizeof(FaceGeo))) != cudaSuccess ||
      (ce = cudaMalloc(&G.colsF, ncol * sizeof(ColGeoF))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f1F, (size_t)n2 * (n1 + 1) * sizeof(FaceGeoF))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f2F, (size_t)(n2 + 1) * n1 * sizeof(FaceGeoF))) != cudaSuccess ||
      (ce = cudaMalloc(&G.f3F, ncol * sizeof(FaceGeoF))) != cudaSuccess ||
      (ce = cudaMalloc(&G.xf_dev, nx * sizeof(double))) != cudaSuccess) {
    err = std::string("geometry allocation failed: ") + cudaGetErrorString(ce);
    free_geometry(G);
    return RAD_ENOMEM;
  }
  std::vector<double> packed;
  packed.insert(packed.end(), G.xf[0].begin(), G.xf[0].end());
  packed.insert(packed.end(), G.xf[1].begin(), G.xf[1].end());
  packed.push_back(G.xf[2].front());
  packed.push_back(G.xf[2][1]);   // uniform x3 spacing: the first cell is representative
  cudaMemcpyAsync(G.xf_dev, packed.data(), nx * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  GeomArgs A;
  A.kind = G.kind;
  A.spin = G.spin;
  A.n1 = n1;
  A.n2 = n2;
  A.n3 = n3;
  A.xf1 = G.xf_dev;
  A.xf2 = G.xf_dev + G.xf[0].size();
  A.xf3 = A.xf2 + G.xf[1].size();
  A.polar_lo = G.bc_lo[1] == RAD_BC_POLAR;
  A.polar_hi = G.bc_hi[1] == RAD_BC_POLAR;
  A.cols = G.cols;
  A.f1 = G.f1;
  A.f2 = G.f2;
  A.f3 = G.f3;
  const int T = 128;
  k_geom_cols<<<(unsigned)((ncol + T - 1) / T), T, 0, ctx->stream>>>(A);
  k_geom_faces<<<(unsigned)(((size_t)n2 * (n1 + 1) + T - 1) / T), T, 0, ctx->stream>>>(A, 0);
  k_geom_faces<<<(unsigned)(((size_t)(n2 + 1) * n1 + T - 1) / T), T, 0, ctx->stream>>>(A, 1);
  k_cols_to_f32<<<(unsigned)((ncol + T - 1) / T), T, 0, ctx->stream>>>(G.cols, G.colsF, (int)ncol);
  k_faces_to_f32<<<(unsigned)(((size_t)n2 * (n1 + 1) + T - 1) / T), T, 0, ctx->stream>>>(G.f1, G.f1F, n2 * (n1 + 1));
  k_faces_to_f32<<<(unsigned)(((size_t)(n2 + 1) * n1 + T - 1) / T), T, 0, ctx->stream>>>(G.f2, G.f2F, (n2 + 1) * n1);
  k_faces_to_f32<<<(unsigned)((ncol + T - 1) / T), T, 0, ctx->stream>>>(G.f3, G.f3F, (int)ncol);
  ce = cudaStreamSynchronize(ctx->stream);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("geometry kernels failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
