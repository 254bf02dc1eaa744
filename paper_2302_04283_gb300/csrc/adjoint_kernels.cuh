// Adjoint of the stage (shared by adjoint.cu and the adjoint_tadj_*.cu
// translation units): the adjoint's argument block, the per-cell CTA
// reductions, and the transposed transport (k_transport_adj, k_tau_grad),
// instantiated per precision and geometry class in adjoint_tadj_*.cu so that
// its many variants (DC/PLM or PPM, with or without the optical-depth
// weighting, three block sizes) compile in parallel.
#pragma once

#include "step_kernel.cuh"

namespace rad {

struct AdjArgs {
  StageArgs s;          // geometry, gas, dims and the stage's coupling step s.dts
  const void *lam;      // coupling adjoint: adjoint of the stage output
  const void *Istar;    // coupling adjoint: saved pre-coupling primitive
  void *mu;             // coupling adjoint output / transport adjoint input
  double *g_aa, *g_as, *g_eta;
  const void *Ilin;     // transport adjoint: state I^{s-1} the operator is linearised at
  void *outA;           // outA (+)= wAf f mu + wAL J_L^T mu
  double wAf, wAL;
  int accA;
  void *outB;           // outB (+)= wBf f mu (nullable)
  double wBf;
  int accB;
  // thermal coupling: adjoint of the stage's output temperature (nullable =
  // 0) and the destinations of wTa lambda_T- ((+)= by accTa) and
  // wTb lambda_T- (=), both nullable
  const double *lamTp;
  double *outTa, *outTb;
  double wTa, wTb;
  int accTa;
  const ColGeo *cols64;  // FP64 column geometry (the thermal reverse sweep runs in FP64)
  // optical-depth weighting: per cell and dimension, the bin sum over the
  // cell's lower face of dL/df * df/d(face alpha_E) (written by
  // k_transport_adj, read by k_tau_grad)
  double *gtau;
  // radiation-dominated substitution: the coupling runs at the substituted
  // velocity (s.u points at it) and writes dL/du [cell][3] here (nullable)
  double *lam_u;
};

// Three-value CTA reduction used per cell: warp reduce-scatter, then every
// thread sums the per-warp partials.  Two barriers.
template <typename R>
__device__ __forceinline__ void cta_sum3(R v0, R v1, R v2, R *buf, int nwarp, int lane, int warp, R out[3]) {
  R s = warp_reduce4(v0, v1, v2, R(0), lane);
  if ((lane & 7) == 0 && lane < 24) buf[warp * 4 + (lane >> 3)] = s;
  __syncthreads();
  out[0] = out[1] = out[2] = R(0);
  for (int w = 0; w < nwarp; ++w) {
    out[0] += buf[w * 4];
    out[1] += buf[w * 4 + 1];
    out[2] += buf[w * 4 + 2];
  }
  __syncthreads();
}

// The same for four values.
template <typename R>
__device__ __forceinline__ void cta_sum4(R v0, R v1, R v2, R v3, R *buf, int nwarp, int lane, int warp, R out[4]) {
  R s = warp_reduce4(v0, v1, v2, v3, lane);
  if ((lane & 7) == 0) buf[warp * 4 + (lane >> 3)] = s;
  __syncthreads();
  out[0] = out[1] = out[2] = out[3] = R(0);
  for (int w = 0; w < nwarp; ++w) {
#pragma unroll
    for (int r = 0; r < 4; ++r) out[r] += buf[w * 4 + r];
  }
  __syncthreads();
}

// Face flux prefactor Delta A n^d n_0 (no 1/dV) and upwind side for one bin.
template <typename Face, typename R>
__device__ __forceinline__ R face_coefA(const Face &F, R x, R y, R z, bool &upR) {
  R na = F.ea[0] + F.ea[1] * x + F.ea[2] * y + F.ea[3] * z;
  R n0 = F.m0[0] + F.m0[1] * x + F.m0[2] * y + F.m0[3] * z;
  upR = na < R(0);
  return F.dA * na * n0;
}

// dphi/d(stencil position) of the upwind face value: stencil values v0 v1 v2,
// phi = v1 +- q(v0, v1, v2) (+ for the left cell, - for the right cell).
template <typename R>
__device__ __forceinline__ void dphi(bool plm, bool right, R v0, R v1, R v2, R d[3]) {
  d[0] = R(0);
  d[1] = R(1);
  d[2] = R(0);
  if (!plm) return;
  R dl = v1 - v0, dr = v2 - v1;
  if (dl * dr > R(0)) {
    R s = dl + dr;
    R is2 = R(1) / (s * s);
    R q0 = -dr * dr * is2, q1 = (dr * dr - dl * dl) * is2, q2 = dl * dl * is2;
    R sg = right ? R(-1) : R(1);
    d[0] = sg * q0;
    d[1] = R(1) + sg * q1;
    d[2] = sg * q2;
  }
}

// Van Leer half-slope q(v0, v1, v2) of the middle cell (0 at extrema).
template <typename R>
__device__ __forceinline__ R half_slope(R v0, R v1, R v2) {
  const R dl = v1 - v0, dr = v2 - v1;
  return dl * dr > R(0) ? dl * dr / (dl + dr) : R(0);
}

// PPM edge value of the middle cell b[2] of five cells (Colella & Woodward
// 1984 on a uniform index grid, as the forward kernel's ppm_states1: limited
// slopes, fourth-order interface values, flattening at extrema, the
// overshoot constraints), its left edge (lft) or right edge, and the
// gradient g[0..4] of that value in b on the active branch.  The expressions
// and branch tests are the forward's, so both take the same branches.
template <typename R>
__device__ __forceinline__ void ppm_edge_grad(const R *b, bool lft, R &val, R g[5]) {
  R sl[3], gs[3][5];
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    R *gm = gs[m - 1];
#pragma unroll
    for (int q = 0; q < 5; ++q) gm[q] = R(0);
    const R dl = b[m] - b[m - 1], dr = b[m + 1] - b[m], dc = R(0.5) * (b[m + 1] - b[m - 1]);
    const R mag = fmin(fabs(dc), fmin(R(2) * fabs(dl), R(2) * fabs(dr)));
    sl[m - 1] = dl * dr > R(0) ? copysign(mag, dc) : R(0);
    if (dl * dr > R(0)) {           // dl, dr and dc share a sign: the slope is dc, 2 dl or 2 dr
      if (fabs(dc) <= fmin(R(2) * fabs(dl), R(2) * fabs(dr))) {
        gm[m + 1] += R(0.5);
        gm[m - 1] -= R(0.5);
      } else if (fabs(dl) <= fabs(dr)) {
        gm[m] += R(2);
        gm[m - 1] -= R(2);
      } else {
        gm[m + 1] += R(2);
        gm[m] -= R(2);
      }
    }
  }
  // interfaces 1|2 (l) and 2|3 (r) of the middle cell
  R l = R(0.5) * (b[1] + b[2]) - (sl[1] - sl[0]) * (R(1) / R(6));
  R r = R(0.5) * (b[2] + b[3]) - (sl[2] - sl[1]) * (R(1) / R(6));
  R gl[5], gr[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    gl[q] = R(0.5) * (R(q == 1) + R(q == 2)) - (gs[1][q] - gs[0][q]) * (R(1) / R(6));
    gr[q] = R(0.5) * (R(q == 2) + R(q == 3)) - (gs[2][q] - gs[1][q]) * (R(1) / R(6));
  }
  const R v = b[2];
  if ((r - v) * (v - l) <= R(0)) {
    l = v;
    r = v;
#pragma unroll
    for (int q = 0; q < 5; ++q) gl[q] = gr[q] = R(q == 2);
  } else {
    const R dlr = r - l, six = dlr * (v - R(0.5) * (l + r)), q6 = dlr * dlr * (R(1) / R(6));
    if (six > q6) {
      l = R(3) * v - R(2) * r;
#pragma unroll
      for (int q = 0; q < 5; ++q) gl[q] = R(3) * R(q == 2) - R(2) * gr[q];
    } else if (-q6 > six) {
      r = R(3) * v - R(2) * l;
#pragma unroll
      for (int q = 0; q < 5; ++q) gr[q] = R(3) * R(q == 2) - R(2) * gl[q];
    }
  }
  val = lft ? l : r;
#pragma unroll
  for (int q = 0; q < 5; ++q) g[q] = lft ? gl[q] : gr[q];
}

// Upwind face state phi and its gradient in the upwind cell's stencil w
// (3 cells for DC / PLM, 5 for PPM): right = the upwind cell is the face's
// right cell (phi is its left edge), else its left cell (phi its right edge).
template <typename R, bool PPM>
__device__ __forceinline__ void edge_grad(bool plm, bool right, const R *w, R &phi, R *d) {
  if (PPM) {
    ppm_edge_grad<R>(w, right, phi, d);
  } else {
    dphi(plm, right, w[0], w[1], w[2], d);
    const R q = plm ? half_slope(w[0], w[1], w[2]) : R(0);
    phi = right ? w[1] - q : w[1] + q;
  }
}

// Transposed transport of one stage (gather form, one thread per target bin).
// PPM: the spatial reconstruction is PPM (each face state depends on the five
// cells around its upwind cell) instead of DC / PLM (three cells).
// AR (with ANG): angular reconstruction, 0 donor cell, 1 PLM along the lines
// of a latitude-longitude grid, 2 minimum-angle planes on a geodesic grid.
template <typename R, bool ANG, int MAXT, bool TAU, bool PPM, int AR>
__global__ void __launch_bounds__(MAXT, sizeof(R) == 8 ? 1 : 1280 / MAXT) k_transport_adj(AdjArgs A) {
  using Col = typename GeoTypes<R>::Col;
  using Face = typename GeoTypes<R>::Face;
  // faces whose upwind stencil can hold this cell: between positions cr and
  // cr + 1 for cr = -HW .. HW - 1 (NF faces); 1/dV and mu at -HW .. HW (NM);
  // the stencils of those faces span -(HW + SW) .. HW + SW (NV values)
  constexpr int SW = PPM ? 2 : 1, HW = SW + 1, NF = 2 * HW, NM = 2 * HW + 1, NV = 2 * (HW + SW) + 1;
  constexpr bool AP = AR == 1, AM = AR == 2;
  const StageArgs &a = A.s;
  const int n = threadIdx.x;
  const bool act = n < a.nang;
  const int nchunk = (a.n3 + a.kc - 1) / a.kc;
  const int col = blockIdx.x / nchunk, chunk = blockIdx.x % nchunk;
  const int i = col % a.n1, j = col / a.n1;
  const int k0 = chunk * a.kc, nc = min(a.kc, a.n3 - k0);
  const long long ncol = (long long)a.n1 * a.n2;
  const long long strideK = ncol * a.nap;
  const bool plm = a.recon == RAD_RECON_PLM;
  const R *Il = (const R *)A.Ilin, *mu = (const R *)A.mu;
  const Col *cols = (const Col *)a.cols;
  const Face *F1 = (const Face *)a.f1, *F2 = (const Face *)a.f2, *F3 = (const Face *)a.f3;
  const int nb_self = act ? n : 0;
  R nh0 = R(0), nh1 = R(0), nh2 = R(0), dOm = R(1);
  if (act) {
    nh0 = (R)a.dir[3 * n];
    nh1 = (R)a.dir[3 * n + 1];
    nh2 = (R)a.dir[3 * n + 2];
    dOm = (R)a.dOmega[n];
  }
  const Col &cg = cols[col];
  const R fconv = cg.n0up * (cg.M[0][0] + cg.M[0][1] * nh0 + cg.M[0][2] * nh1 + cg.M[0][3] * nh2);
  const int nperm = act ? a.perm[n] : 0;

  // per dimension: the NF faces between positions (cr, cr+1), cr = -HW..HW-1,
  // and 1/dV at positions -HW..HW (0 for ghosts of non-periodic dimensions)
  int nd = a.ndim;
  R cA[3][NF], ivd[3][NM];
  bool uR[3][NF], fex[3][NF];
  int N[3] = {a.n1, a.n2, a.n3};
  int y[3] = {i, j, 0};
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < NF; ++t) {
      cA[d][t] = R(0);
      uR[d][t] = false;
      fex[d][t] = false;
    }
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < NM; ++t) ivd[d][t] = R(0);
  for (int d = 0; d < nd && d < 2; ++d) {
    const bool per = a.bc_lo[d] == RAD_BC_PERIODIC;
    for (int t = 0; t < NM; ++t) {
      int p = y[d] + t - HW;
      bool ghost = p < 0 || p >= N[d];
      if (ghost && !per) continue;
      int pp = ((p % N[d]) + N[d]) % N[d];
      int c2 = d == 0 ? j * a.n1 + pp : pp * a.n1 + i;
      ivd[d][t] = cols[c2].invdV;
    }
    for (int t = 0; t < NF; ++t) {
      int c = y[d] + t - HW;         // face between cells c and c+1, face index c+1
      bool ex = per || (c >= -1 && c <= N[d] - 1);
      fex[d][t] = ex && act;
      if (!fex[d][t]) continue;
      int fi = per ? ((c + 1) % N[d] + N[d]) % N[d] : c + 1;
      const Face &F = d == 0 ? F1[j * (a.n1 + 1) + fi] : F2[fi * a.n1 + i];
      bool u;
      cA[d][t] = face_coefA(F, nh0, nh1, nh2, u);
      uR[d][t] = u;
    }
  }
  if (nd >= 3) {
    bool u;
    R c3 = act ? face_coefA(F3[col], nh0, nh1, nh2, u) : R(0);
    for (int t = 0; t < NF; ++t) {
      cA[2][t] = c3;
      uR[2][t] = act ? u : false;
    }
    for (int t = 0; t < NM; ++t) ivd[2][t] = cg.invdV;
  }
  // angular PLM (AP): the sides whose flux depends on this bin -- its own
  // sides (it is the upwind or the downwind cell) and the sides whose upwind
  // line reconstruction takes it as the cell behind -- with, per side, the
  // prefactor P = len (V . nu) n_0 of Eq. flux_angle for this column, the
  // cells p, q of the side and the upwind, downwind and behind cells
  constexpr int NE = AP ? kMaxSlots + kMaxBehind : 1;
  R ap_P[NE];
  int ap_e[NE], ap_p[NE], ap_q[NE], ap_u[NE], ap_d[NE], ap_b[NE];
  auto edge_P = [&](int e, bool &upp) -> R {
      const double *eg = a.edge_geo + 8 * e;
      const R x = (R)eg[0], yv = (R)eg[1], z = (R)eg[2], len = (R)eg[6];
      const R pr[10] = {R(1), x, yv, z, x * x, x * yv, x * z, yv * yv, yv * z, z * z};
      R q0 = R(0), q1 = R(0), q2 = R(0);
      for (int p = 0; p < 10; ++p) {
        q0 += cg.K[0][p] * pr[p];
        q1 += cg.K[1][p] * pr[p];
        q2 += cg.K[2][p] * pr[p];
      }
      const R sp = -((R)eg[3] * q0 + (R)eg[4] * q1 + (R)eg[5] * q2);
      upp = sp >= R(0);                       // upwind: p (ties to p, as the forward)
      return len * sp * (cg.M[0][0] + cg.M[0][1] * x + cg.M[0][2] * yv + cg.M[0][3] * z);
  };
  // MAPR (AM): every side's prefactor and upwind side for this column
  __shared__ R amP[AM ? 3 * kMaxBinsStep : 1];
  __shared__ unsigned char amUp[AM ? 3 * kMaxBinsStep : 1];
  if (AM) {
    for (int e = threadIdx.x; e < a.n_edge; e += blockDim.x) {
      bool upp;
      amP[e] = edge_P(e, upp);
      amUp[e] = upp;
    }
    __syncthreads();
  }
  if (AP) {
    for (int s = 0; s < NE; ++s) {
      ap_P[s] = R(0);
      ap_e[s] = -1;
      ap_p[s] = ap_q[s] = ap_u[s] = ap_d[s] = ap_b[s] = nb_self;
      int e = -1, side = -1;
      if (s < kMaxSlots) {
        if (act && a.slot_nbr[6 * n + s] >= 0) e = a.slot_edge[6 * n + s];
      } else {
        const int code = act ? a.line_behind[kMaxBehind * n + (s - kMaxSlots)] : -1;
        if (code >= 0) {
          e = code >> 1;
          side = code & 1;
        }
      }
      if (e < 0) continue;
      bool upp;
      const R P = edge_P(e, upp);
      if (side >= 0 && upp != (side == 0)) continue;     // the reconstruction is from the other cell
      const int p = a.edge_pq[2 * e], q = a.edge_pq[2 * e + 1];
      ap_P[s] = P;
      ap_e[s] = e;
      ap_p[s] = p;
      ap_q[s] = q;
      ap_u[s] = upp ? p : q;
      ap_d[s] = upp ? q : p;
      ap_b[s] = a.edge_line[2 * e + (upp ? 0 : 1)];
    }
    // a side that is both one of this bin's own and one it is behind of
    // (no lat/long grid has one) counts once
    for (int s = kMaxSlots; s < NE; ++s)
      for (int s2 = 0; s2 < kMaxSlots; ++s2)
        if (ap_e[s] >= 0 && ap_e[s] == ap_e[s2]) ap_e[s] = -1;
  }
  // angular: transposed coefficients
  R at_self = R(0), at_nb[kMaxSlots];
  int nb_m[kMaxSlots];
  if (ANG && !AP && !AM) {
    R self = R(0);
    for (int s = 0; s < kMaxSlots; ++s) {
      at_nb[s] = R(0);
      nb_m[s] = nb_self;
      int m = act ? a.slot_nbr[6 * n + s] : -1;
      if (m < 0) continue;
      nb_m[s] = m;
      int e = a.slot_edge[6 * n + s];
      const double *eg = a.edge_geo + 8 * e;
      R x = (R)eg[0], yv = (R)eg[1], z = (R)eg[2], v0 = (R)eg[3], v1 = (R)eg[4], v2 = (R)eg[5], len = (R)eg[6];
      R pr[10] = {R(1), x, yv, z, x * x, x * yv, x * z, yv * yv, yv * z, z * z};
      R q0 = R(0), q1 = R(0), q2 = R(0);
      for (int p = 0; p < 10; ++p) {
        q0 += cg.K[0][p] * pr[p];
        q1 += cg.K[1][p] * pr[p];
        q2 += cg.K[2][p] * pr[p];
      }
      R sp = -(v0 * q0 + v1 * q1 + v2 * q2);
      R n0e = cg.M[0][0] + cg.M[0][1] * x + cg.M[0][2] * yv + cg.M[0][3] * z;
      R P = len * sp * n0e;
      R PL = sp >= R(0) ? P : R(0), PR = sp >= R(0) ? R(0) : P;
      R dOm_m = (R)a.dOmega[m];
      // forward: divA_n gets (n == p ? PL : -PR) / dOm_n from I_n and
      // (n == p ? PR : -PL) / dOm_n from I_m; the transpose gathers what
      // divA_m takes from I_n
      if (a.edge_pq[2 * e] == n) {
        self += PL / dOm;
        at_nb[s] = -PL / dOm_m;
      } else {
        self -= PR / dOm;
        at_nb[s] = PR / dOm_m;
      }
    }
    at_self = act ? self : R(0);
  }
  // neighbour addressing along x1 / x2 (periodic wrap, outflow clamp; polar
  // positions are handled separately).  A polar position further from the
  // pole than the line is long mirrors to no row (the index returned is then
  // outside [0, N)); no face in use reaches it, and callers load nothing there.
  auto src_idx = [&](int d, int p, bool &ghost, bool &polar) -> int {
    ghost = p < 0 || p >= N[d];
    polar = false;
    if (!ghost) return p;
    int lo = a.bc_lo[d], hi = a.bc_hi[d];
    if (p < 0) {
      if (lo == RAD_BC_PERIODIC) return ((p % N[d]) + N[d]) % N[d];
      if (lo == RAD_BC_OUTFLOW) return 0;
      polar = true;
      return -1 - p;
    }
    if (hi == RAD_BC_PERIODIC) return p % N[d];
    if (hi == RAD_BC_OUTFLOW) return N[d] - 1;
    polar = true;
    return 2 * N[d] - 1 - p;
  };
  R *outA = (R *)A.outA, *outB = (R *)A.outB;
  constexpr bool tauw = TAU;                       // optical-depth weighting (a.tau_const > 0)
  __shared__ R tbuf[TAU ? (MAXT / 32) * 4 : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = 0; c < nc; ++c) {
    const int k = k0 + c;
    y[2] = k;
    R gt[3] = {R(0), R(0), R(0)};   // lower-face sums of this bin (optical-depth weighting)
    auto addr = [&](int ii, int jj, int kk, int bin) -> long long {
      return (long long)kk * strideK + ((long long)jj * a.n1 + ii) * a.nap + bin;
    };
    const long long eown = addr(i, j, k, nb_self);
    const R mu0 = act ? mu[eown] : R(0);
    R lam = R(0);
    for (int d = 0; d < nd; ++d) {
      // stencil values at positions -(HW+SW)..HW+SW and mu at -HW..HW along d
      R v[NV], mm[NM];
      bool match[NV];
      for (int t = 0; t < NV; ++t) {
        bool ghost, pol;
        int p = y[d] + t - (HW + SW);
        int q = src_idx(d, p, ghost, pol);
        int ii = i, jj = j, kk = k, bin = nb_self;
        if (d == 0) ii = q;
        if (d == 1) jj = q;
        if (d == 2) kk = q;
        if (pol) {
          kk = a.n3 > 1 ? (k + a.n3 / 2) % a.n3 : k;
          bin = nperm;
        }
        const bool inr = q >= 0 && q < N[d];
        v[t] = act && inr ? Il[addr(ii, jj, kk, bin)] : R(0);
        match[t] = inr && !pol && (q == y[d]);
        if (t >= SW && t < SW + NM)
          mm[t - SW] = (ghost && a.bc_lo[d] != RAD_BC_PERIODIC) || !act ? R(0) : mu[addr(ii, jj, kk, bin)];
      }
      // optical-depth weighting: 1 / n^0bar of the cells at positions -HW..HW
      // and, per face t (positions t - HW | t - HW + 1), d_t and df/d(alpha_E)
      R nbi[NM], fdt[NF], dfa[NF];
      if (tauw) {
        R ux5[NM], uy5[NM], uz5[NM], ae5[NM];
        for (int t = 0; t < NM; ++t) {
          bool ghost, pol;
          int q = src_idx(d, y[d] + t - HW, ghost, pol);
          if (q < 0 || q >= N[d]) q = y[d];        // no such row: the faces next to it are not in use
          int ii = i, jj = j, kk = k;
          if (d == 0) ii = q;
          if (d == 1) jj = q;
          if (d == 2) kk = q;
          if (pol) kk = a.n3 > 1 ? (k + a.n3 / 2) % a.n3 : k;
          const long long cell = (long long)kk * ncol + (long long)jj * a.n1 + ii;
          ux5[t] = (R)a.u[3 * cell];
          uy5[t] = (R)a.u[3 * cell + 1];
          uz5[t] = (R)a.u[3 * cell + 2];
          ae5[t] = (R)a.aa[cell] + (R)a.as[cell];
          const R u0 = sqrt(R(1) + ux5[t] * ux5[t] + uy5[t] * uy5[t] + uz5[t] * uz5[t]);
          nbi[t] = R(1) / (u0 - (ux5[t] * nh0 + uy5[t] * nh1 + uz5[t] * nh2));
        }
        for (int t = 0; t < NF; ++t) {
          const R fx = R(0.5) * (ux5[t] + ux5[t + 1]), fy = R(0.5) * (uy5[t] + uy5[t + 1]),
                  fz = R(0.5) * (uz5[t] + uz5[t + 1]);
          const R u0F = sqrt(R(1) + fx * fx + fy * fy + fz * fz);
          const R tdt = (R)a.tau_const * (R)a.dt / u0F;           // dtau / d(face alpha_E)
          const R tq = tdt * (R(0.5) * (ae5[t] + ae5[t + 1]));
          const R f = -rexpm1(-tq * tq);
          fdt[t] = R(0.5) * f * (nbi[t] - nbi[t + 1]);
          dfa[t] = R(2) * tq * (R(1) - f) * tdt;                     // df/dtau dtau/d(face alpha_E)
        }
      }
      const bool per = a.bc_lo[d] == RAD_BC_PERIODIC;
      for (int t = 0; t < NF; ++t) {
        if (d == 2) {   // x3 faces exist unless they lie beyond a non-periodic boundary
          const int cf = k + t - HW;
          fex[2][t] = act && (per || (cf >= -1 && cf <= a.n3 - 1));
        }
        if (!fex[d][t]) continue;
        if (per && N[d] < NF) {   // a short periodic line: count each physical face once
          bool seen = false;
#pragma unroll 1
          for (int t2 = 0; t2 < t; ++t2) seen |= (t - t2) % N[d] == 0;
          if (seen) continue;
        }
        // face between positions cr = t - HW and cr + 1 (mu / 1/dV index t, t + 1)
        R lphi = -cA[d][t] * ivd[d][t] * mm[t] + cA[d][t] * ivd[d][t + 1] * mm[t + 1];
        const bool right = uR[d][t];
        const int s0 = t + (right ? 1 : 0);   // window index of the upwind stencil's first cell
        R ph, dd[2 * SW + 1];
        edge_grad<R, PPM>(plm, right, v + s0, ph, dd);
        if (tauw) {
          if (t == HW - 1)   // this cell's lower face: the flux's derivative in f
            gt[d] = lphi * ph * (right ? R(-0.5) : R(0.5)) * (nbi[HW - 1] - nbi[HW]) * dfa[HW - 1];
          lphi *= right ? R(1) - fdt[t] : R(1) + fdt[t];
        }
        R g = R(0);
        for (int u = 0; u < 2 * SW + 1; ++u)
          if (match[s0 + u]) g += dd[u];
        lam += lphi * g;
      }
    }
    // polar: this cell is a ghost row of the mirrored column (k + n3/2, the
    // mirrored bin) -- row -1 - j beyond theta = 0, row 2 n2 - 1 - j beyond
    // theta = pi -- and the upwind stencils of that column's faces next to
    // the pole (faces of non-zero area: 1 .. n2 - 1) can reach it
    if (nd >= 2 && act) {
      const int kk = a.n3 > 1 ? (k + a.n3 / 2) % a.n3 : k;
      const int bp = nperm;                         // bin of the mirrored direction
      const R px = (R)a.dir[3 * bp], py = (R)a.dir[3 * bp + 1], pz = (R)a.dir[3 * bp + 2];
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        if ((side ? a.bc_hi[1] : a.bc_lo[1]) != RAD_BC_POLAR) continue;
        const int gr = side ? 2 * a.n2 - 1 - j : -1 - j;     // this cell's row in the mirrored column
        const int f0 = side ? max(1, gr - SW) : 1, f1 = side ? a.n2 - 1 : min(a.n2 - 1, gr + SW + 1);
#pragma unroll 1
        for (int fi = f0; fi <= f1; ++fi) {                  // face between rows fi - 1 and fi
          bool u;
          const R cAf = face_coefA(F2[fi * a.n1 + i], px, py, pz, u);
          const int ur = u ? fi : fi - 1;                    // upwind row
          if (gr < ur - SW || gr > ur + SW) continue;
          const int jl = fi - 1, jr = fi;
          R lphi = -cAf * cols[jl * a.n1 + i].invdV * mu[addr(i, jl, kk, bp)] +
                   cAf * cols[jr * a.n1 + i].invdV * mu[addr(i, jr, kk, bp)];
          if (tauw) {   // the factor of this face for bin bp
            const long long cl = (long long)kk * ncol + (long long)jl * a.n1 + i, cr = cl + a.n1;
            const R uxl = (R)a.u[3 * cl], uyl = (R)a.u[3 * cl + 1], uzl = (R)a.u[3 * cl + 2];
            const R uxr = (R)a.u[3 * cr], uyr = (R)a.u[3 * cr + 1], uzr = (R)a.u[3 * cr + 2];
            const R fx = R(0.5) * (uxl + uxr), fy = R(0.5) * (uyl + uyr), fz = R(0.5) * (uzl + uzr);
            const R tq = (R)a.tau_const * (R(0.5) * ((R)a.aa[cl] + (R)a.as[cl] + (R)a.aa[cr] + (R)a.as[cr])) *
                         (R)a.dt / sqrt(R(1) + fx * fx + fy * fy + fz * fz);
            const R f = -rexpm1(-tq * tq);
            const R nl = R(1) / (sqrt(R(1) + uxl * uxl + uyl * uyl + uzl * uzl) - (uxl * px + uyl * py + uzl * pz));
            const R nr = R(1) / (sqrt(R(1) + uxr * uxr + uyr * uyr + uzr * uzr) - (uxr * px + uyr * py + uzr * pz));
            const R df = R(0.5) * f * (nl - nr);
            lphi *= u ? R(1) - df : R(1) + df;
          }
          // the upwind stencil, rows ur - SW .. ur + SW of the mirrored
          // column; rows beyond a pole are rows of this column, own bin
          R sv[2 * SW + 1];
          for (int q = 0; q < 2 * SW + 1; ++q) {
            const int r = ur - SW + q;
            if (r < 0) sv[q] = Il[addr(i, -1 - r, k, nb_self)];
            else if (r >= a.n2) sv[q] = Il[addr(i, 2 * a.n2 - 1 - r, k, nb_self)];
            else sv[q] = Il[addr(i, r, kk, bp)];
          }
          R ph, dd[2 * SW + 1];
          edge_grad<R, PPM>(plm, u, sv, ph, dd);
          lam += lphi * dd[gr - (ur - SW)];
        }
      }
    }
    if (ANG && !AP && !AM) {
      R ga = at_self * mu0;
      for (int s = 0; s < kMaxSlots; ++s) ga += at_nb[s] * mu[addr(i, j, k, nb_m[s])];
      lam -= ga;
    }
    if (AP) {
      // the side's flux F = P (I_u + q(I_b, I_u, I_d)) leaves p and enters q:
      // d<mu, L>/dI = -P (mu_p / dOmega_p - mu_q / dOmega_q) dF/dI, through
      // every role (behind, upwind, downwind) this bin plays on the side
      for (int s = 0; s < NE; ++s) {
        if (ap_e[s] < 0) continue;
        const int p = ap_p[s], q = ap_q[s];
        const R lphiA = -ap_P[s] * (mu[addr(i, j, k, p)] / (R)a.dOmega[p] - mu[addr(i, j, k, q)] / (R)a.dOmega[q]);
        R d[3];
        dphi(true, false, Il[addr(i, j, k, ap_b[s])], Il[addr(i, j, k, ap_u[s])], Il[addr(i, j, k, ap_d[s])], d);
        lam += lphiA * ((ap_b[s] == n ? d[0] : R(0)) + (ap_u[s] == n ? d[1] : R(0)) + (ap_d[s] == n ? d[2] : R(0)));
      }
    }
    if (AM && act) {
      // a side's upwind value is I_u + g_u . x = I_u + w_a (I_a - I_u) +
      // w_b (I_b - I_u), (w_a, w_b) = A^T x with A the inverse of u's chosen
      // plane (cells a, b) on its active branch; this bin enters the sides
      // of u = itself or a neighbour whose chosen plane holds it
#pragma unroll 1
      for (int ci = 0; ci <= kMaxSlots; ++ci) {
        const int u = ci == 0 ? n : a.slot_nbr[6 * n + ci - 1];
        if (u < 0) continue;
        const int *nbc = a.mapr_nb + 6 * u;
        const double *mi = a.mapr_minv + 24 * u;
        const R Iu = Il[addr(i, j, k, u)];
        R dl[6];
        for (int q = 0; q < 6; ++q) dl[q] = nbc[q] >= 0 ? Il[addr(i, j, k, nbc[q])] - Iu : R(0);
        const int K = nbc[5] >= 0 ? 6 : 5;
        int best = 0;
        R bq = R(0);
        for (int q = 0; q < K; ++q) {
          const int q2 = q + 1 == K ? 0 : q + 1;
          const R x = (R)mi[4 * q] * dl[q] + (R)mi[4 * q + 1] * dl[q2];
          const R y = (R)mi[4 * q + 2] * dl[q] + (R)mi[4 * q + 3] * dl[q2];
          const R qq = x * x + y * y;
          if (q == 0 || qq < bq) {
            bq = qq;
            best = q;
          }
        }
        const int b2 = best + 1 == K ? 0 : best + 1;
        const int ma = nbc[best], mb = nbc[b2];
        if (n != u && n != ma && n != mb) continue;
        const double *m4 = mi + 4 * best;
#pragma unroll 1
        for (int s = 0; s < kMaxSlots; ++s) {
          if (a.slot_nbr[6 * u + s] < 0) continue;
          const int e = a.slot_edge[6 * u + s];
          const int p = a.edge_pq[2 * e], q = a.edge_pq[2 * e + 1];
          if ((u == p) != (amUp[e] != 0)) continue;          // u is not upwind of this side
          const double *xs = a.mapr_xo + 12 * u + 2 * s;
          const R wa = (R)(m4[0] * xs[0] + m4[2] * xs[1]), wb = (R)(m4[1] * xs[0] + m4[3] * xs[1]);
          const R dv = (n == u ? R(1) - wa - wb : R(0)) + (n == ma ? wa : R(0)) + (n == mb ? wb : R(0));
          lam += -amP[e] * (mu[addr(i, j, k, p)] / (R)a.dOmega[p] - mu[addr(i, j, k, q)] / (R)a.dOmega[q]) * dv;
        }
      }
    }
    if (tauw) {
      R gs[3];
      cta_sum3(gt[0], gt[1], gt[2], tbuf, nwarp, lane, warp, gs);
      if (threadIdx.x == 0) {
        const long long cell = (long long)k * ncol + (long long)j * a.n1 + i;
        for (int d = 0; d < 3; ++d) A.gtau[3 * cell + d] = (double)gs[d];
      }
    }
    if (act) {
      R ra = (R)A.wAf * fconv * mu0 + (R)A.wAL * lam;
      outA[eown] = A.accA ? outA[eown] + ra : ra;
      if (outB) {
        R rb = (R)A.wBf * fconv * mu0;
        outB[eown] = A.accB ? outB[eown] + rb : rb;
      }
    }
  }
}

namespace {

// dL/dalpha_a and dL/dalpha_s through the optical-depth weighting, one thread
// per cell: the sums of its lower faces (its own gtau) and of its upper faces
// (the next cell's gtau along each dimension, wrapping where periodic; a
// non-periodic upper boundary face carries none: outflow copies the
// velocity, so d = 0 there, and polar faces have zero area).  The face
// alpha_E is the mean of its two cells', hence the 1/2; w = the stage's
// weight of the transport operator (beta dt).
__global__ void k_tau_grad(const double *gtau, int n1, int n2, int n3, int ndim, int per0, int per1, int per2,
                           double w, double *g_aa, double *g_as) {
  const long long ncell = (long long)n1 * n2 * n3;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  const int N[3] = {n1, n2, n3}, per[3] = {per0, per1, per2};
  const int x[3] = {(int)(cell % n1), (int)((cell / n1) % n2), (int)(cell / ((long long)n1 * n2))};
  const long long stride[3] = {1, n1, (long long)n1 * n2};
  double g = 0.0;
  for (int d = 0; d < ndim; ++d) {
    g += gtau[3 * cell + d];
    if (x[d] + 1 < N[d]) g += gtau[3 * (cell + stride[d]) + d];
    else if (per[d]) g += gtau[3 * (cell - (long long)(N[d] - 1) * stride[d]) + d];
  }
  const double ge = 0.5 * w * g;
  g_aa[cell] += ge;
  g_as[cell] += ge;
}

}  // namespace

template <typename R, bool ANG, int AR, int MAXT>
void launch_tadj(const AdjArgs &A, bool tau, bool ppm, dim3 grid, int threads, cudaStream_t st) {
  if (ppm)
    tau ? k_transport_adj<R, ANG, MAXT, true, true, AR><<<grid, threads, 0, st>>>(A)
        : k_transport_adj<R, ANG, MAXT, false, true, AR><<<grid, threads, 0, st>>>(A);
  else
    tau ? k_transport_adj<R, ANG, MAXT, true, false, AR><<<grid, threads, 0, st>>>(A)
        : k_transport_adj<R, ANG, MAXT, false, false, AR><<<grid, threads, 0, st>>>(A);
}

// AR: angular reconstruction (curved space only): 0 donor cell, 1 line PLM, 2 MAPR
template <typename R, bool ANG, int AR = 0>
cudaError_t launch_transport_adj(const AdjArgs &A, cudaStream_t st) {
  int threads = (A.s.nap + 31) / 32 * 32;
  int nchunk = (A.s.n3 + A.s.kc - 1) / A.s.kc;
  dim3 grid((unsigned)((long long)A.s.n1 * A.s.n2 * nchunk));
  const bool tau = A.s.tau_const > 0.0, ppm = A.s.recon == RAD_RECON_PPM;
  if (threads <= 256) launch_tadj<R, ANG, AR, 256>(A, tau, ppm, grid, threads, st);
  else if (threads <= 512) launch_tadj<R, ANG, AR, 512>(A, tau, ppm, grid, threads, st);
  else launch_tadj<R, ANG, AR, 1024>(A, tau, ppm, grid, threads, st);
  if (tau) {
    const StageArgs &a = A.s;
    const long long ncell = (long long)a.n1 * a.n2 * a.n3;
    k_tau_grad<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(
        A.gtau, a.n1, a.n2, a.n3, a.ndim, a.bc_lo[0] == RAD_BC_PERIODIC, a.bc_lo[1] == RAD_BC_PERIODIC,
        a.bc_lo[2] == RAD_BC_PERIODIC, A.wAL, A.g_aa, A.g_as);
  }
  return cudaGetLastError();
}

// Explicitly instantiated in adjoint_tadj_<precision>_<flat|ang|angplm|angmapr>.cu.
extern template cudaError_t launch_transport_adj<float, false>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<float, true>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<double, false>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<double, true>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<float, true, 1>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<double, true, 1>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<float, true, 2>(const AdjArgs &, cudaStream_t);
extern template cudaError_t launch_transport_adj<double, true, 2>(const AdjArgs &, cudaStream_t);

}  // namespace rad
