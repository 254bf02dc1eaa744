// Fused stage kernel of the radiation update: spatial reconstruction and
// upwind fluxes (Secs. 2.3-2.4, Eq. flux_space), geodesic angular fluxes
// (Eq. flux_angle, Sec. 2.6), the RK stage combination of Eq.
// radiation_integral, the locally implicit coupling (Sec. 2.5) and the
// n0crit guard (Sec. 2.4).
//
// Work decomposition: one CTA per (i, j) column and chunk of at most
// kMaxChunk cells along x3; one thread per angle bin.  The metrics are
// x3-independent, so every geometric prefactor of a bin is built once per
// CTA (in the working precision, from the per-column tables) and kept in
// registers while the thread walks the chunk along x3 with the x3 stencil in
// a sliding register window.  x1 / x2 neighbours are coalesced row loads.
// Boundary conditions are applied by index mapping (no ghost cells):
// periodic wrap, outflow clamp, and the polar map (theta -> -theta,
// phi -> phi + pi, bin n -> perm[n]).
//
// Three phases per CTA:
//   A  for each cell: fluxes, stage combination, primitive I* (written to the
//      output row), and the three angle sums of the coupling (A1 - Ebar, A2,
//      Ebar; a warp reduce-scatter, per-warp partials in shared memory);
//   B  one thread per cell sums the warp partials and solves its quartic for
//      T+ in FP64 (all cells of the chunk in parallel);
//   C  for each cell: the implicit update of every bin from I* (re-read from
//      the output row, still in L2) and the source S of phase B, and the four
//      sums of (I+ - I*) n^A dOmega that give the gas source;
//   D  one thread per cell turns those sums into -dR^0_mu.
#pragma once

#include <cuda_runtime.h>

#include "rad_internal.h"

namespace rad {

constexpr int kNRedA = 3;   // phase A sums
constexpr int kNRedC = 4;   // phase C sums
constexpr int kMaxChunk = 32;
constexpr double kFourPi = 12.566370614359172953850573533118;

struct StageArgs {
  const void *Iprev;      // I^{s-1}: neighbours and own bin (read-only)
  const void *I0;         // I^0 (own bin, stage 2)
  void *Iout;
  void *Istar;            // optional copy of the pre-coupling primitive I* (adjoint recompute)
  const double *T0, *T1;  // T^0, and T^1 for stage 2
  double *Tout;
  const double *rho, *u, *aa, *as, *eta;
  double *src;
  int stage2;             // 0: U* = U^0 + dt L;  1: U* = U^0/2 + (U^1 + dt L)/2
  double dt, dts;         // full step and coupling step (dt, then dt/2)
  int n1, n2, n3, nap, nang, ndim, kc;
  int bc_lo[3], bc_hi[3];
  const void *cols;       // ColGeo or ColGeoF
  const void *f1, *f2, *f3;
  const double *dir, *dOmega, *edge_geo;
  const int *perm, *slot_nbr, *slot_edge, *edge_pq;
  int recon, mode, zero_guard;
  double n0crit, a_rad, gamma;
  int *err;
};

StageArgs make_stage_args(rad_ctx *ctx, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src);
cudaError_t launch_stage(const StageArgs &a, bool f32, bool ang, cudaStream_t st);

template <typename R> struct GeoTypes;
template <> struct GeoTypes<double> { using Col = ColGeo; using Face = FaceGeo; };
template <> struct GeoTypes<float> { using Col = ColGeoF; using Face = FaceGeoF; };

template <typename R> __device__ __forceinline__ R fdiv(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }

// PLM half-slope q = dl dr / (dl + dr) if dl dr > 0 else 0 (van Leer 1974).
template <typename R>
__device__ __forceinline__ R vl_half(R x, R y, R z) {
  R dl = y - x, dr = z - y;
  R prod = dl * dr;
  return prod > R(0) ? fdiv(prod, dl + dr) : R(0);
}

// Upwind value at the face between cells b and c of the stencil a b | c d:
// the right cell's reconstruction if upR, else the left cell's.
template <typename R>
__device__ __forceinline__ R face_val(bool upR, bool plm, R a, R b, R c, R d) {
  if (!plm) return upR ? c : b;
  R x = upR ? b : a, y = upR ? c : b, z = upR ? d : c;
  R q = vl_half(x, y, z);
  return upR ? y - q : y + q;
}

// Positive root of B4 T^4 + B1 T + B0 (B4 >= 0, B1 > 0, B0 <= 0).  f is
// convex and increasing for T >= 0, so Newton from the upper bound
// min(-B0/B1, (-B0/B4)^(1/4)) (the root lies within a factor 2 below it)
// decreases monotonically onto the root.  FP32 iterations get close
// cheaply; FP64 iterations finish (the slope may be the FP32 one: Newton
// with a slope accurate to 1e-7 still gains seven digits per iteration).
__device__ __forceinline__ double quartic_root(double B4, double B1, double B0, bool full64, bool &ok) {
  if (!(B1 > 0.0) || !(B4 >= 0.0) || !(B0 <= 0.0)) {
    ok = false;
    return 0.0;
  }
  if (B0 == 0.0) return 0.0;
  double T = -B0 / B1;
  if (B4 == 0.0) return T;
  T = fmin(T, sqrt(sqrt(-B0 / B4)));
  if (full64) {
    for (int it = 0; it < 80; ++it) {
      double t2 = T * T;
      double f = fma(fma(B4, t2 * T, B1), T, B0);
      double fp = fma(4.0 * B4, t2 * T, B1);
      double Tn = T - f / fp;
      if (!(Tn < T)) return T;
      if (T - Tn <= 1e-16 * T) return Tn;
      T = Tn;
    }
    ok = false;
    return T;
  }
  float tf = (float)T, b4f = (float)B4, b1f = (float)B1, b0f = (float)B0;
  for (int it = 0; it < 40; ++it) {
    float t2 = tf * tf;
    float f = fmaf(fmaf(b4f, t2 * tf, b1f), tf, b0f);
    float fp = fmaf(4.0f * b4f, t2 * tf, b1f);
    float tn = tf - __fdividef(f, fp);
    if (!(tn < tf) || !(tn > 0.0f)) break;
    tf = tn;
  }
  T = (double)tf;
  for (int it = 0; it < 3; ++it) {
    double t2 = T * T;
    double f = fma(fma(B4, t2 * T, B1), T, B0);
    float fp = fmaf(4.0f * b4f, (float)(t2 * T), b1f);
    T = T - f * (double)(1.0f / fp);
  }
  if (!(T > 0.0) || !isfinite(T)) ok = false;
  return T;
}

// Warp reduce-scatter of four values: on return the lane holds the warp sum
// of value ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1); lanes 0, 8, 16, 24
// hold values 0, 1, 2, 3.  Six shuffles instead of twenty.
template <typename R>
__device__ __forceinline__ R warp_reduce4(R v0, R v1, R v2, R v3, int lane) {
  const bool hi16 = lane & 16;
  R a0 = hi16 ? v2 : v0, a1 = hi16 ? v3 : v1;
  R s0 = hi16 ? v0 : v2, s1 = hi16 ? v1 : v3;
  a0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  a1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool hi8 = lane & 8;
  R b = hi8 ? a1 : a0;
  b += __shfl_xor_sync(0xffffffffu, hi8 ? a0 : a1, 8);
  b += __shfl_xor_sync(0xffffffffu, b, 4);
  b += __shfl_xor_sync(0xffffffffu, b, 2);
  b += __shfl_xor_sync(0xffffffffu, b, 1);
  return b;
}

struct Nbr {
  long long col_off;  // (jj * n1 + ii) * nap
  int kshift;         // 0 or n3 / 2 (polar)
  int polar;          // read bin perm[n]
};

__device__ __forceinline__ int wrap_idx(int x, int n, int bc_lo, int bc_hi, int &polar) {
  polar = 0;
  if (x < 0) {
    if (bc_lo == RAD_BC_PERIODIC) return ((x % n) + n) % n;
    if (bc_lo == RAD_BC_OUTFLOW) return 0;
    polar = 1;
    return -1 - x;
  }
  if (x >= n) {
    if (bc_hi == RAD_BC_PERIODIC) return x % n;
    if (bc_hi == RAD_BC_OUTFLOW) return n - 1;
    polar = 1;
    return 2 * n - 1 - x;
  }
  return x;
}

// Shared-memory footprint (bytes) of k_stage for a block of `threads`.
template <typename R, bool ANG>
__host__ __device__ constexpr size_t stage_smem(int threads, int nap) {
  return (size_t)kMaxChunk * 4 * sizeof(R)                          // gas: ux uy uz alphaE
         + (size_t)kMaxChunk * sizeof(R)                            // u^0hat
         + (size_t)kMaxChunk * (threads / 32) * kNRedC * sizeof(R)  // per-warp partial sums
         + (size_t)kMaxChunk * kNRedC * sizeof(R)                   // cell sums
         + (size_t)kMaxChunk * sizeof(R)                            // S per cell
         + (ANG ? (size_t)2 * nap * sizeof(R) : 0);                 // own-cell rows
}

template <typename R, bool ANG, int MAXT>
__global__ void __launch_bounds__(MAXT) k_stage(StageArgs a) {
  using Col = typename GeoTypes<R>::Col;
  using Face = typename GeoTypes<R>::Face;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = threadIdx.x;
  const int nwarp = blockDim.x >> 5;
  const int lane = n & 31, warp = n >> 5;
  const bool act = n < a.nang;
  const int nchunk = (a.n3 + a.kc - 1) / a.kc;
  const int col = blockIdx.x / nchunk;
  const int chunk = blockIdx.x % nchunk;
  const int i = col % a.n1, j = col / a.n1;
  const int k0 = chunk * a.kc;
  const int nc = min(a.kc, a.n3 - k0);
  const long long strideK = (long long)a.n1 * a.n2 * a.nap;
  const long long ncol = (long long)a.n1 * a.n2;
  const R *Ip = (const R *)a.Iprev;
  const R *I0 = (const R *)a.I0;
  R *Io = (R *)a.Iout;
  const bool plm = a.recon == RAD_RECON_PLM;
  const bool couple = a.mode != RAD_COUPLE_NONE;

  R *sgas = (R *)smem_raw;                                 // [kMaxChunk][4]
  R *su0 = sgas + kMaxChunk * 4;                            // [kMaxChunk]
  R *red = su0 + kMaxChunk;                                 // [kMaxChunk][nwarp][kNRedC]
  R *sums = red + kMaxChunk * nwarp * kNRedC;               // [kMaxChunk][kNRedC]
  R *Sc = sums + kMaxChunk * kNRedC;                        // [kMaxChunk]
  R *rows = Sc + kMaxChunk;                                 // [2][nap]

  // ---- gas state of the chunk (one conversion per cell)
  for (int c = n; c < nc; c += blockDim.x) {
    long long cell = (long long)(k0 + c) * ncol + col;
    if (couple) {
      double ux = a.u[3 * cell], uy = a.u[3 * cell + 1], uz = a.u[3 * cell + 2];
      sgas[4 * c + 0] = (R)ux;
      sgas[4 * c + 1] = (R)uy;
      sgas[4 * c + 2] = (R)uz;
      sgas[4 * c + 3] = (R)(a.aa[cell] + a.as[cell]);
      su0[c] = (R)sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    }
  }

  // ---- per-bin prefactors of this column
  const Col &cg = ((const Col *)a.cols)[col];
  R nh0 = R(0), nh1 = R(0), nh2 = R(0), dOm = R(1);
  if (act) {
    nh0 = (R)a.dir[3 * n];
    nh1 = (R)a.dir[3 * n + 1];
    nh2 = (R)a.dir[3 * n + 2];
    dOm = (R)a.dOmega[n];
  }
  const R n0up = cg.n0up;
  const R nlow0 = cg.M[0][0] + cg.M[0][1] * nh0 + cg.M[0][2] * nh1 + cg.M[0][3] * nh2;
  const R fconv = n0up * nlow0;                          // U = n^0 n_0 I
  const bool guard = act && a.zero_guard && fabs((double)nlow0) < a.n0crit;
  const R inv_f = act ? R(1) / fconv : R(0);
  const R invdV = cg.invdV;
  auto fcoef = [&](const Face &F, bool &upR) -> R {
    R na = F.ea[0] + F.ea[1] * nh0 + F.ea[2] * nh1 + F.ea[3] * nh2;
    R n0 = F.m0[0] + F.m0[1] * nh0 + F.m0[2] * nh1 + F.m0[3] * nh2;
    upR = na < R(0);
    return F.dA * na * n0 * invdV;
  };
  R cm[3] = {R(0), R(0), R(0)}, cp[3] = {R(0), R(0), R(0)};
  bool um[3] = {false, false, false}, up[3] = {false, false, false};
  if (act) {
    const Face *F1 = (const Face *)a.f1, *F2 = (const Face *)a.f2, *F3 = (const Face *)a.f3;
    cm[0] = fcoef(F1[j * (a.n1 + 1) + i], um[0]);
    cp[0] = fcoef(F1[j * (a.n1 + 1) + i + 1], up[0]);
    if (a.ndim >= 2) {
      cm[1] = fcoef(F2[j * a.n1 + i], um[1]);
      cp[1] = fcoef(F2[(j + 1) * a.n1 + i], up[1]);
    }
    if (a.ndim >= 3) {
      cm[2] = fcoef(F3[col], um[2]);
      cp[2] = cm[2];
      up[2] = um[2];
    }
  }
  // angular flux: divA_n = a_self I_n + sum_s a_nb[s] I_{m_s}
  R a_self = R(0);
  R a_nb[kMaxSlots];
  int nb_m[kMaxSlots];
  if (ANG) {
    R self = R(0);
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      a_nb[s] = R(0);
      nb_m[s] = act ? n : 0;
      int m = act ? a.slot_nbr[6 * n + s] : -1;
      if (m < 0) continue;
      nb_m[s] = m;
      int e = a.slot_edge[6 * n + s];
      const double *eg = a.edge_geo + 8 * e;
      R x = (R)eg[0], y = (R)eg[1], z = (R)eg[2], v0 = (R)eg[3], v1 = (R)eg[4], v2 = (R)eg[5], len = (R)eg[6];
      R pr[10] = {R(1), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
      R q0 = R(0), q1 = R(0), q2 = R(0);
#pragma unroll
      for (int p = 0; p < 10; ++p) {
        q0 += cg.K[0][p] * pr[p];
        q1 += cg.K[1][p] * pr[p];
        q2 += cg.K[2][p] * pr[p];
      }
      R sp = -(v0 * q0 + v1 * q1 + v2 * q2);           // V . nu (nu is normal to n_e)
      R n0e = cg.M[0][0] + cg.M[0][1] * x + cg.M[0][2] * y + cg.M[0][3] * z;
      R P = len * sp * n0e;
      R PL = sp >= R(0) ? P : R(0), PR = sp >= R(0) ? R(0) : P;
      if (a.edge_pq[2 * e] == n) {
        self += PL;
        a_nb[s] = PR / dOm;
      } else {
        self -= PR;
        a_nb[s] = -PL / dOm;
      }
    }
    a_self = act ? self / dOm : R(0);
  }
  // x1 / x2 neighbours of this column
  Nbr nx[4], ny[4];
  const int offs[4] = {-2, -1, 1, 2};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int pol;
    int ii = wrap_idx(i + offs[t], a.n1, a.bc_lo[0], a.bc_hi[0], pol);
    nx[t].col_off = ((long long)j * a.n1 + ii) * a.nap;
    nx[t].kshift = 0;
    nx[t].polar = 0;
    int jj = j;
    pol = 0;
    if (a.ndim >= 2) jj = wrap_idx(j + offs[t], a.n2, a.bc_lo[1], a.bc_hi[1], pol);
    ny[t].col_off = ((long long)jj * a.n1 + i) * a.nap;
    ny[t].kshift = pol ? a.n3 / 2 : 0;
    ny[t].polar = pol;
  }
  const int nperm = act ? a.perm[n] : 0;
  const int nself = act ? n : 0;
  const long long own = (long long)col * a.nap + nself;
  auto kidx = [&](int k) {
    int pol;
    return wrap_idx(k, a.n3, a.bc_lo[2], a.bc_hi[2], pol);
  };
  auto ld_nb = [&](const Nbr &nb, int k) -> R {
    int kk = k + nb.kshift;
    if (kk >= a.n3) kk -= a.n3;
    return __ldg(Ip + (long long)kk * strideK + nb.col_off + (nb.polar ? nperm : nself));
  };
  const R dtR = (R)a.dt, dts = (R)a.dts;
  const R c2pre = dts / R(kFourPi);
  __syncthreads();   // gas staged

  // ---- phase A
  R win[5];
  const bool d3 = a.ndim >= 3;
  if (d3) {
#pragma unroll
    for (int t = 0; t < 4; ++t) win[t + 1] = __ldg(Ip + (long long)kidx(k0 - 2 + t) * strideK + own);
  }
  for (int c = 0; c < nc; ++c) {
    const int k = k0 + c;
    R zc, sx = R(0);
    if (d3) {
#pragma unroll
      for (int t = 0; t < 4; ++t) win[t] = win[t + 1];
      win[4] = __ldg(Ip + (long long)kidx(k + 2) * strideK + own);
      zc = win[2];
      R lo = face_val(um[2], plm, win[0], win[1], win[2], win[3]);
      R hi = face_val(up[2], plm, win[1], win[2], win[3], win[4]);
      sx = cp[2] * hi - cm[2] * lo;
    } else {
      zc = __ldg(Ip + (long long)k * strideK + own);
    }
    {
      R m2 = ld_nb(nx[0], k), m1 = ld_nb(nx[1], k), p1 = ld_nb(nx[2], k), p2 = ld_nb(nx[3], k);
      sx += cp[0] * face_val(up[0], plm, m1, zc, p1, p2) - cm[0] * face_val(um[0], plm, m2, m1, zc, p1);
    }
    if (a.ndim >= 2) {
      R m2 = ld_nb(ny[0], k), m1 = ld_nb(ny[1], k), p1 = ld_nb(ny[2], k), p2 = ld_nb(ny[3], k);
      sx += cp[1] * face_val(up[1], plm, m1, zc, p1, p2) - cm[1] * face_val(um[1], plm, m2, m1, zc, p1);
    }
    R divA = R(0);
    if (ANG) {
      R *row = rows + (c & 1) * a.nap;
      if (n < a.nap) row[n] = zc;
      __syncthreads();
      divA = a_self * zc;
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) divA += a_nb[s] * row[nb_m[s]];
    }
    const R L = -(sx + divA);
    const R Uprev = fconv * zc;
    R Us;
    if (a.stage2) {
      R U0 = fconv * (act ? I0[(long long)k * strideK + own] : R(0));
      Us = R(0.5) * U0 + R(0.5) * (Uprev + dtR * L);
    } else {
      Us = Uprev + dtR * L;
    }
    const R Is = (guard || !act) ? R(0) : Us * inv_f;
    if (act) {
      Io[(long long)k * strideK + own] = Is;
      if (a.Istar) ((R *)a.Istar)[(long long)k * strideK + own] = Is;
    }
    if (couple) {
      const R ux = sgas[4 * c], uy = sgas[4 * c + 1], uz = sgas[4 * c + 2], aE = sgas[4 * c + 3];
      const R nb = su0[c] - (ux * nh0 + uy * nh1 + uz * nh2);
      const R rden = fdiv(R(1), n0up + nb * aE * dts);
      const R w = Is * nb * nb * dOm;                      // Ibar dOmega_bar
      // A1 - Ebar = sum (c1 - 1) Ibar dOmega_bar, A2' = sum dOmega / (n^0bar den), Ebar
      R v0 = act ? -(nb * aE * dts) * rden * w : R(0);
      R v1 = act ? fdiv(dOm * rden, nb) : R(0);
      R v2 = act ? w : R(0);
      R s = warp_reduce4(v0, v1, v2, R(0), lane);
      if ((lane & 7) == 0 && lane < 24) red[(c * nwarp + warp) * kNRedC + (lane >> 3)] = s;
    }
  }

  if (couple) {
    __syncthreads();
    // ---- phase B: one thread per cell
    for (int t = n; t < nc * kNRedA; t += blockDim.x) {
      int c = t / kNRedA, r = t % kNRedA;
      R s = R(0);
      for (int w = 0; w < nwarp; ++w) s += red[(c * nwarp + w) * kNRedC + r];
      sums[c * kNRedC + r] = s;
    }
    __syncthreads();
    if (n < nc) {
      const int c = n, k = k0 + c;
      const long long cell = (long long)k * ncol + col;
      const R *rs = sums + c * kNRedC;
      const double D = (double)rs[0], A2 = a.dts / kFourPi * (double)rs[1], Em = (double)rs[2];
      const double Tst = a.stage2 ? 0.5 * (a.T0[cell] + a.T1[cell]) : a.T0[cell];
      const double aa = a.aa[cell], as = a.as[cell];
      double S, Tp = Tst;
      bool ok = true;
      if (a.mode == RAD_COUPLE_THERMAL) {
        const double cv = a.rho[cell] / (a.gamma - 1.0);
        const double B4 = A2 * aa * a.a_rad;
        const double B1 = cv * (1.0 - A2 * as);
        const double B0 = D + A2 * as * Em - B1 * Tst;   // A1 - B1 T- - (1 - A2 alpha_s) Ebar-
        Tp = quartic_root(B4, B1, B0, sizeof(R) == 8, ok);
        const double Ep = Em - cv * (Tp - Tst);
        const double T2 = Tp * Tp;
        S = aa * a.a_rad * T2 * T2 + as * Ep;
      } else {
        const double eta = a.eta[cell];
        const double den = 1.0 - A2 * as;
        ok = den > 0.0;
        const double Ep = (D + Em + kFourPi * A2 * eta) / den;
        S = kFourPi * eta + as * Ep;
      }
      if (!ok || !isfinite(Tp) || !isfinite(S)) atomicOr(a.err, kErrNoConv);
      Sc[c] = (R)S;
      a.Tout[cell] = Tp;
    }
    __syncthreads();
  } else if (n < nc) {
    const long long cell = (long long)(k0 + n) * ncol + col;
    a.Tout[cell] = a.stage2 ? 0.5 * (a.T0[cell] + a.T1[cell]) : a.T0[cell];
    if (a.src && !a.stage2) {
      for (int m = 0; m < 4; ++m) a.src[4 * cell + m] = 0.0;
    }
  }

  // ---- phase C: implicit update of every bin
  bool bad = false;
  const bool want_src = couple && a.src;
  for (int c = 0; c < nc; ++c) {
    const int k = k0 + c;
    R *po = Io + (long long)k * strideK + own;
    R Is = act ? *po : R(0);
    R out = Is;
    if (couple) {
      const R ux = sgas[4 * c], uy = sgas[4 * c + 1], uz = sgas[4 * c + 2], aE = sgas[4 * c + 3];
      const R nb = su0[c] - (ux * nh0 + uy * nh1 + uz * nh2);
      const R rden = fdiv(R(1), n0up + nb * aE * dts);
      const R c2n = fdiv(c2pre * rden, nb * nb * nb);     // c2 / (n^0bar)^4
      out = n0up * rden * Is + c2n * Sc[c];
    }
    if (want_src) {
      // gas source: sums of (I+ - I*) n^A dOmega (taken before the guard)
      R d = act ? (out - Is) * dOm : R(0);
      R s = warp_reduce4(d, d * nh0, d * nh1, d * nh2, lane);
      if ((lane & 7) == 0) red[(c * nwarp + warp) * kNRedC + (lane >> 3)] = s;
    }
    if (guard) out = R(0);
    if (act) {
      *po = out;
      bad |= !isfinite(out);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonFinite);
  if (want_src) {
    // ---- phase D: -dR^0_mu with dR^0_mu = n^0 M[mu][A] sum (I+ - I*) n^A dOmega
    __syncthreads();
    if (n < nc) {
      const int c = n;
      const long long cell = (long long)(k0 + c) * ncol + col;
      R xs[4];
#pragma unroll
      for (int A = 0; A < 4; ++A) {
        R t = R(0);
        for (int w = 0; w < nwarp; ++w) t += red[(c * nwarp + w) * kNRedC + A];
        xs[A] = t;
      }
      double *sp = a.src + 4 * cell;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        R dR = n0up * (cg.M[m][0] * xs[0] + cg.M[m][1] * xs[1] + cg.M[m][2] * xs[2] + cg.M[m][3] * xs[3]);
        sp[m] = a.stage2 ? sp[m] - (double)dR : -0.5 * (double)dR;
      }
    }
  }
}

}  // namespace rad
