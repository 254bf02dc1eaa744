// Fused stage kernel of the radiation update: spatial reconstruction and
// upwind fluxes (Secs. 2.3-2.4, Eq. flux_space), geodesic angular fluxes
// (Eq. flux_angle, Sec. 2.6), the RK stage combination of Eq.
// radiation_integral, the locally implicit coupling (Sec. 2.5) and the
// n0crit guard (Sec. 2.4).
//
// Work decomposition: one CTA per (i, j) column and chunk of at most
// kMaxChunk cells along x3.  The metrics are x3-independent, so every
// geometric prefactor of a bin is built once per CTA (in the working
// precision, from the per-column tables) and kept in registers while the CTA
// walks its chunk along x3.  Each consumer thread owns two adjacent angle
// bins (8- or 16-byte shared-memory accesses, packed FP32x2 arithmetic).
//
// Data movement: one extra producer warp streams every cell's stencil rows
// from global memory into a ring of 2-4 stages in shared memory with 1D bulk
// TMA copies (cp.async.bulk ... mbarrier::complete_tx).  The rows of a cell
// are the contiguous x1 block i-2..i+2 (one copy; five at a wrapped or
// clamped boundary), the four x2 rows j-2, j-1, j+1, j+2, the own column's
// row at k+2 (the x3 stencil is a sliding register window with its limiter
// slopes carried along) and, in stage 2, the own row of I^0.  A "full"
// mbarrier per ring stage counts the bytes in; an "empty" mbarrier per stage
// collects one arrival per consumer warp before the producer refills it, so
// no CTA-wide barrier is taken per cell.  Every wait is bounded and sets an
// error bit on timeout.
// Boundary conditions are applied by index mapping (no ghost cells):
// periodic wrap, outflow clamp, and the polar map (theta -> -theta,
// phi -> phi + pi, bin n -> perm[n]).
//
// Phases per CTA:
//   A  for each cell: fluxes, stage combination, primitive I* (kept in shared
//      memory for the chunk), and the three angle sums of the coupling
//      (A1 - Ebar, A2, Ebar; a warp reduce-scatter, per-warp partials in
//      shared memory);
//   B  one thread per cell sums the warp partials and solves its quartic for
//      T+ in FP64 (all cells of the chunk in parallel);
//   C  for each cell: the implicit update of every bin from I* and the source
//      S of phase B, written to the output row, and the four sums of
//      (I+ - I*) n^A dOmega that give the gas source;
//   D  one thread per cell turns those sums into -dR^0_mu.
#pragma once

#include <cuda_runtime.h>

#include <string>

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
  int sign_pairs;         // bins 2t, 2t + 1 have no direction component of opposite sign
  int depth;                       // stages of the shared-memory ring (2..kMaxStages)
  int bc_lo[3], bc_hi[3];
  const void *cols;       // ColGeo or ColGeoF
  const ColGeo *cols64;   // the FP64 columns (the separate coupling kernel of the rad_dom option)
  const void *f1, *f2, *f3;
  const double *dir, *dOmega, *edge_geo;
  const int *perm, *slot_nbr, *slot_edge, *edge_pq;
  const int *edge_line;    // latitude-longitude grids: cell behind p, cell beyond q of each side
  const int *line_behind;  // latitude-longitude grids: per bin, the sides it is the cell behind of (adjoint)
  int n_edge;              // sides of the angle grid
  const int *mapr_nb;      // geodesic grids: neighbours in cyclic order, plane inverses, side midpoints
  const double *mapr_minv, *mapr_xo, *mapr_xn;
  int recon_ang;           // RAD_RECON_DC or RAD_RECON_PLM (angular fluxes)
  int recon, mode, zero_guard;
  double n0crit, a_rad, gamma;
  double inv_gm1;          // 1 / (gamma - 1)
  double tau_const;       // C of the optical-depth flux weighting (0: free streaming)
  int *err;
  const void *halo[6];     // ghost rows of faces shared with other blocks: face (d, side) at 2 d + side
  const void *divF;        // multigroup: this group's frequency divergence [cell][nap] (null: gray)
};

StageArgs make_stage_args(rad_ctx *ctx, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src);
cudaError_t launch_stage(const StageArgs &a, bool f32, bool ang, cudaStream_t st);
// One precision / geometry class of stage launches (explicitly instantiated in
// stage_<precision>_<flat|ang>.cu, one translation unit each).
// NAP > 0 fixes the padded row length (a.nap) at compile time; 0 reads it
// from the arguments; NAP < 0 fixes it at -NAP in a kernel that also reads
// halo rows and a frequency divergence (those, like NAP = 0, do).
// AR: angular reconstruction (curved space): 0 donor cell, 1 PLM along the
// lines of a latitude-longitude grid, 2 minimum-angle planes on a geodesic grid.
template <typename R, bool ANG, int AR = 0, int NAP = 0>
cudaError_t launch_stage_rp(const StageArgs &a, cudaStream_t st);
// Padded rows of the level-4, 6 and 8 geodesic grids (162, 362, 642 bins):
// the FP32 kernels have variants with these row lengths fixed (the flat-space
// kernel at level 4, the curved-space one at all three), where the constant
// row stride folds the ring and chunk addressing into immediates.
constexpr int kNapGeo4 = 164, kNapGeo6 = 364, kNapGeo8 = 644;
// RAD_OK, or RAD_EUNSUPPORTED with a message when a stage launch of this
// grid / bin count cannot be formed (element count, shared memory, threads).
int check_stage(const StageArgs &a, bool f32, std::string &err);
// Coupling with the radiation-dominated velocity substitution (raddom.cu):
// I* in s.Iout -> I+, T- (Tm) -> T+ (Tout), the gas source of stage s.stage2.
cudaError_t launch_couple_rd(const StageArgs &s, bool f32, const double *Tm, double *Tout, cudaStream_t st);
// The substitution of the rad_dom option for the adjoint (raddom.cu): mode 0
// writes the substituted velocity of every cell from the saved I* and T-,
// mode 1 takes dL/du_sub back to mu, T- (outTa / outTb, weighted) and the
// opacity gradients.
cudaError_t launch_rd_sub(int mode, const StageArgs &s, bool f32, const void *Istar, const double *Tm,
                          double *usub, const double *lam_u, void *mu, double *g_aa, double *g_as, double *outTa,
                          double wTa, double *outTb, double wTb, cudaStream_t st);

template <typename R> struct GeoTypes;
template <> struct GeoTypes<double> { using Col = ColGeo; using Face = FaceGeo; };
template <> struct GeoTypes<float> { using Col = ColGeoF; using Face = FaceGeoF; };

template <typename R> __device__ __forceinline__ R fdiv(R a, R b) { return a / b; }
__device__ __forceinline__ double rexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float rexpm1(float x) { return expm1f(x); }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
// hardware approximate reciprocal (one MUFU op, within an ulp or so); the FP32
// path's stated tolerance covers it
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// FP64 reciprocal: the hardware approximation r refined by one third-order
// step.  With e = 1 - x r, 1/x = r / (1 - e) = r (1 + e + e^2 + ...); keeping
// three terms, r <- r + r (e + e^2), turns a relative error eps of r into
// about eps^3.  The approximation's eps measured on GB300 is below 1e-6
// (2^-19.9 over 4M random x across the exponent range), so one step lands
// within an ulp of the correctly rounded 1/x (equal to it for 99.97 % of
// those x; two Newton-Raphson steps matched it everywhere).  Three FP64
// operations instead of the four of two Newton-Raphson steps, and far
// cheaper on the FP64 pipe than a correctly rounded division; far inside the
// FP64 path's 1e-12 tolerance.  x = 0 gives a non-finite result (as 1/x
// does); callers discard it.
__device__ __forceinline__ double rcp_newton(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
// prod > 0 for the limiter: the FP32 compare, or in FP64 an integer test of
// the high word (sign, exponent and the top of the mantissa), which keeps the
// compare off the FP64 pipe.  A positive FP64 value whose high word is zero
// (below 2^-1022 x 2^-20) counts as zero, so its limited slope, smaller
// still, becomes zero.
__device__ __forceinline__ bool pos_for_limiter(float v) { return v > 0.0f; }
__device__ __forceinline__ bool pos_for_limiter(double v) { return __double2hiint(v) > 0; }

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
// decreases monotonically onto the root.  The FP32 path gets close in FP32
// and finishes with FP64 steps (Newton with a slope accurate to 1e-7 still
// gains seven digits per step), falling back to the FP64 iteration when the
// FP64 residual is not small; the FP64 path iterates in FP64 throughout.
// guess > 0 (the temperature before the coupling, usually close to the
// root): one Newton step from it first.  f is convex, so from either side
// the step lands at or above the root; inside the bracket it replaces the
// upper bound as the start of the monotone iteration (a few steps instead
// of a few tens when the coupling changes T little).
__device__ __forceinline__ double quartic_root(double B4, double B1, double B0, bool full64, bool &ok,
                                               double guess = -1.0) {
  if (!(B1 > 0.0) || !(B4 >= 0.0) || !(B0 <= 0.0)) {
    ok = false;
    return 0.0;
  }
  if (B0 == 0.0) return 0.0;
  if (B4 == 0.0) return -B0 / B1;
  if (!full64) {
    // FP32 bracket and Newton iterations, then two FP64 Newton steps with the
    // FP32 slope; the FP64 residual decides whether the full FP64 solve below
    // is still needed (it is not, unless the FP32 range was exceeded)
    const float b4f = (float)B4, b1f = (float)B1, b0f = (float)B0;
    float tf = fminf(-b0f / b1f, sqrtf(sqrtf(-b0f / b4f)));
    if (guess > 0.0) {
      const float g = (float)guess, g3 = g * g * g;
      const float tg = g - __fdividef(fmaf(fmaf(b4f, g3, b1f), g, b0f), fmaf(4.0f * b4f, g3, b1f));
      if (tg > 0.0f && tg < tf) tf = tg;
    }
    for (int it = 0; it < 40; ++it) {
      const float t2 = tf * tf;
      const float f = fmaf(fmaf(b4f, t2 * tf, b1f), tf, b0f);
      const float fp = fmaf(4.0f * b4f, t2 * tf, b1f);
      const float tn = tf - __fdividef(f, fp);
      if (!(tn < tf) || !(tn > 0.0f)) break;
      tf = tn;
    }
    double T = (double)tf, f = 0.0;
    for (int it = 0; it < 2; ++it) {
      const double t2 = T * T;
      f = fma(fma(B4, t2 * T, B1), T, B0);
      const float fp = fmaf(4.0f * b4f, (float)(t2 * T), b1f);
      T = T - f * (double)(1.0f / fp);
    }
    const double t2 = T * T;
    f = fma(fma(B4, t2 * T, B1), T, B0);
    if (T > 0.0 && isfinite(T) && fabs(f) <= 1e-9 * -B0) return T;
  }
  // FP64: Newton from the upper bound decreases monotonically onto the root
  double T = fmin(-B0 / B1, sqrt(sqrt(-B0 / B4)));
  if (guess > 0.0) {
    const double g3 = guess * guess * guess;
    const double tg = guess - fma(fma(B4, g3, B1), guess, B0) / fma(4.0 * B4, g3, B1);
    if (tg > 0.0 && tg < T) T = tg;
  }
  for (int it = 0; it < 80; ++it) {
    const double t2 = T * T;
    const double f = fma(fma(B4, t2 * T, B1), T, B0);
    const double fp = fma(4.0 * B4, t2 * T, B1);
    const double Tn = T - f / fp;
    if (!(Tn < T)) return T;
    if (T - Tn <= 1e-16 * T) return Tn;
    T = Tn;
  }
  ok = false;
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

// Warp reduce-scatter of eight values: on return lane l holds the warp sum
// of value (l >> 2) & 7, so lanes 0, 4, ..., 28 hold values 0 .. 7.  Nine
// shuffles (two warp_reduce4 calls take twelve) in one five-deep chain.
template <typename R>
__device__ __forceinline__ R warp_reduce8(const R (&v)[8], int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8, hi4 = lane & 4;
  R a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = hi16 ? v[4 + k] : v[k];
    a[k] += __shfl_xor_sync(0xffffffffu, hi16 ? v[k] : v[4 + k], 16);
  }
  R b[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    b[k] = hi8 ? a[2 + k] : a[k];
    b[k] += __shfl_xor_sync(0xffffffffu, hi8 ? a[k] : a[2 + k], 8);
  }
  R c = hi4 ? b[1] : b[0];
  c += __shfl_xor_sync(0xffffffffu, hi4 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// The same for sixteen values: lane l ends with the sum of value (l >> 1)
// & 15, so lanes 0, 2, ..., 30 hold values 0 .. 15 (sixteen shuffles).
template <typename R>
__device__ __forceinline__ R warp_reduce16(const R (&v)[16], int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8, hi4 = lane & 4, hi2 = lane & 2;
  R a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = hi16 ? v[8 + k] : v[k];
    a[k] += __shfl_xor_sync(0xffffffffu, hi16 ? v[k] : v[8 + k], 16);
  }
  R b[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b[k] = hi8 ? a[4 + k] : a[k];
    b[k] += __shfl_xor_sync(0xffffffffu, hi8 ? a[k] : a[4 + k], 8);
  }
  R c[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    c[k] = hi4 ? b[2 + k] : b[k];
    c[k] += __shfl_xor_sync(0xffffffffu, hi4 ? b[k] : b[2 + k], 4);
  }
  R d = hi2 ? c[1] : c[0];
  d += __shfl_xor_sync(0xffffffffu, hi2 ? c[0] : c[1], 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// The same for thirty-two values: lane l ends with the sum of value l
// (thirty-one shuffles).
template <typename R>
__device__ __forceinline__ R warp_reduce32(const R (&v)[32], int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8, hi4 = lane & 4, hi2 = lane & 2, hi1 = lane & 1;
  R a[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = hi16 ? v[16 + k] : v[k];
    a[k] += __shfl_xor_sync(0xffffffffu, hi16 ? v[k] : v[16 + k], 16);
  }
  R b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    b[k] = hi8 ? a[8 + k] : a[k];
    b[k] += __shfl_xor_sync(0xffffffffu, hi8 ? a[k] : a[8 + k], 8);
  }
  R c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c[k] = hi4 ? b[4 + k] : b[k];
    c[k] += __shfl_xor_sync(0xffffffffu, hi4 ? b[k] : b[4 + k], 4);
  }
  R d[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    d[k] = hi2 ? c[2 + k] : c[k];
    d[k] += __shfl_xor_sync(0xffffffffu, hi2 ? c[k] : c[2 + k], 2);
  }
  R e = hi1 ? d[1] : d[0];
  e += __shfl_xor_sync(0xffffffffu, hi1 ? d[0] : d[1], 1);
  return e;
}

// A cell's staged gas values (ux, uy, uz, alpha_E, u0) read with two
// vector loads from its 8-element row, returned through a small array.
template <typename R> struct GasRow { R v[8]; };
__device__ __forceinline__ GasRow<float> gas_load(const float *row) {
  GasRow<float> g;
  const float4 a = *(const float4 *)row, b = *(const float4 *)(row + 4);
  g.v[0] = a.x; g.v[1] = a.y; g.v[2] = a.z; g.v[3] = a.w;
  g.v[4] = b.x; g.v[5] = b.y; g.v[6] = b.z; g.v[7] = b.w;
  return g;
}
__device__ __forceinline__ GasRow<double> gas_load(const double *row) {
  GasRow<double> g;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 a = *(const double2 *)(row + 2 * q);
    g.v[2 * q] = a.x;
    g.v[2 * q + 1] = a.y;
  }
  return g;
}

struct Nbr {
  long long col_off;  // (jj * n1 + ii) * nap
  int kshift;         // 0 or n3 / 2 (polar)
  int polar;          // read bin perm[n]
};

// Index of the cell a stencil position x (possibly outside 0..n-1) reads.
// kind: 0 a cell of this block (periodic wrap, outflow clamp), 1 the polar
// mirror (theta -> -theta: the caller shifts phi by pi and permutes the
// bins), 2 / 3 a ghost of a lower / upper face shared with another block
// (RAD_BC_HALO): the value returned is then the ghost layer, 0 next to the
// face.
// HALO false: kernels that never see a shared face (kind is 0 or 1).
template <bool HALO = true>
__device__ __forceinline__ int wrap_idx(int x, int n, int bc_lo, int bc_hi, int &kind) {
  kind = 0;
  if (x < 0) {
    if (bc_lo == RAD_BC_PERIODIC) return ((x % n) + n) % n;
    if (bc_lo == RAD_BC_OUTFLOW) return 0;
    kind = (HALO && bc_lo == RAD_BC_HALO) ? 2 : 1;
    return -1 - x;
  }
  if (x >= n) {
    if (bc_hi == RAD_BC_PERIODIC) return x % n;
    if (bc_hi == RAD_BC_OUTFLOW) return n - 1;
    if (HALO && bc_hi == RAD_BC_HALO) {
      kind = 3;
      return x - n;
    }
    kind = 1;
    return 2 * n - 1 - x;
  }
  return x;
}

// Row of ghost layer `layer` of face (d, side) in that face's halo buffer
// (rad_halo_pack's layout): [layer][k][j] for x1 faces, [layer][k][i] for x2
// faces, [layer][j][i] for x3 faces, rows of nap elements.
template <typename R>
__device__ __forceinline__ const R *halo_row(const void *const *halo, int n1, int n2, int n3, int d, int side,
                                             int layer, int i, int j, int k, int nap) {
  const R *b = (const R *)halo[2 * d + side];
  size_t r;
  if (d == 0) r = ((size_t)layer * n3 + k) * n2 + j;
  else if (d == 1) r = ((size_t)layer * n3 + k) * n1 + i;
  else r = ((size_t)layer * n2 + j) * n1 + i;
  return b + r * nap;
}

// ---------------------------------------------------------------- pairs
// Two bins per thread.  For float the arithmetic uses the packed FP32x2
// instructions of sm_100+ (one instruction for both bins); for double it is
// two scalar operations.
template <typename R> struct P2;
template <> struct P2<float> {
  using V = float2;
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  // approximate reciprocal (MUFU, ~1 ulp): the FP32 path's stated tolerance allows it
  static __device__ __forceinline__ V rcp(V a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
};
template <> struct P2<double> {
  using V = double2;
  static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
  static __device__ __forceinline__ V rcp(V a) { return make_double2(rcp_newton(a.x), rcp_newton(a.y)); }
};

// van Leer half-slopes of a pair: q = dl dr / (dl + dr) if dl dr > 0, else 0.
template <typename R>
__device__ __forceinline__ typename P2<R>::V vl2(typename P2<R>::V x, typename P2<R>::V y, typename P2<R>::V z) {
  using P = P2<R>;
  auto dl = P::sub(y, x), dr = P::sub(z, y);
  auto prod = P::mul(dl, dr);
  auto s = P::add(dl, dr);
  // both quotients are formed unconditionally and the select discards the
  // ones of non-positive products (including 0/0), so no branch is taken
  const auto q = P::mul(prod, P::rcp(s));                      // one (packed) multiply by reciprocals
  return P::mk(pos_for_limiter(prod.x) ? q.x : R(0), pos_for_limiter(prod.y) ? q.y : R(0));
}

template <typename R>
__device__ __forceinline__ typename P2<R>::V sel2(bool cx, bool cy, typename P2<R>::V a, typename P2<R>::V b) {
  return P2<R>::mk(cx ? a.x : b.x, cy ? a.y : b.y);
}

// Upwind face values of the lower (m1|c) and upper (c|p1) faces from the
// three half-slopes q(m2,m1,c), q(m1,c,p1), q(c,p1,p2) of the pair.
template <typename R>
__device__ __forceinline__ typename P2<R>::V face_div(unsigned um, unsigned up, typename P2<R>::V cm,
                                                    typename P2<R>::V cp, typename P2<R>::V m1,
                                                    typename P2<R>::V c, typename P2<R>::V p1,
                                                    typename P2<R>::V qm, typename P2<R>::V qc,
                                                    typename P2<R>::V qp) {
  using P = P2<R>;
  const bool umx = um & 1, umy = um & 2, upx = up & 1, upy = up & 2;
  auto lo = P::add(sel2<R>(umx, umy, c, m1), sel2<R>(umx, umy, P::mk(-qc.x, -qc.y), qm));
  auto hi = P::add(sel2<R>(upx, upy, p1, c), sel2<R>(upx, upy, P::mk(-qp.x, -qp.y), qc));
  return P::sub(P::mul(cp, hi), P::mul(cm, lo));
}

// PPM (Colella & Woodward 1984) face states of the two faces of the middle
// cell of a seven-cell line a[0..6] (a[3] = own), on a uniform index grid:
// limited slopes (the smallest of the central difference and twice the
// one-sided ones, zero at extrema), fourth-order interface values from them,
// and the two monotonicity constraints on every cell's parabola.  Returns the
// left / right states of the lower face (cells 2 | 3) and the upper face
// (cells 3 | 4).
template <typename R>
__device__ __forceinline__ void ppm_states1(const R (&a)[7], R &loL, R &loR, R &hiL, R &hiR) {
  R sl[7];
#pragma unroll
  for (int m = 1; m <= 5; ++m) {
    const R dl = a[m] - a[m - 1], dr = a[m + 1] - a[m], dc = R(0.5) * (a[m + 1] - a[m - 1]);
    const R mag = fmin(fabs(dc), fmin(R(2) * fabs(dl), R(2) * fabs(dr)));
    sl[m] = dl * dr > R(0) ? copysign(mag, dc) : R(0);
  }
  R e[6];                                      // e[m]: interface between cells m and m + 1
#pragma unroll
  for (int m = 1; m <= 4; ++m) e[m] = R(0.5) * (a[m] + a[m + 1]) - (sl[m + 1] - sl[m]) * (R(1) / R(6));
  R aL[5], aR[5];
#pragma unroll
  for (int c = 2; c <= 4; ++c) {
    R l = e[c - 1], r = e[c];
    const R v = a[c];
    if ((r - v) * (v - l) <= R(0)) {
      l = v;
      r = v;
    } else {
      const R dlr = r - l, six = dlr * (v - R(0.5) * (l + r)), q = dlr * dlr * (R(1) / R(6));
      if (six > q) l = R(3) * v - R(2) * r;
      else if (-q > six) r = R(3) * v - R(2) * l;
    }
    aL[c] = l;
    aR[c] = r;
  }
  loL = aR[2];
  loR = aL[3];
  hiL = aR[3];
  hiR = aL[4];
}

template <typename R>
__device__ __forceinline__ void ppm_states(const typename P2<R>::V (&a)[7], typename P2<R>::V &loL,
                                           typename P2<R>::V &loR, typename P2<R>::V &hiL,
                                           typename P2<R>::V &hiR) {
  R ax[7], ay[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    ax[q] = a[q].x;
    ay[q] = a[q].y;
  }
  ppm_states1<R>(ax, loL.x, loR.x, hiL.x, hiR.x);
  ppm_states1<R>(ay, loL.y, loR.y, hiL.y, hiR.y);
}

// face_div in weighted form (no selects in the cell loop): ncmL / ncmR are
// -(lower-face coefficient) where the upwind state is the left / right one
// and 0 otherwise, cpL / cpR likewise for the upper face, and
//   div = ncmL (m1 + qm) + ncmR (c - qc) + cpL (c + qc) + cpR (p1 - qp)
// is evaluated with the own cell's terms gathered: A = ncmR + cpL multiplies
// c and B = cpL - ncmR the own slope qc (six multiply-adds instead of four
// sums and four multiply-adds).
template <typename R>
__device__ __forceinline__ typename P2<R>::V face_div_g(typename P2<R>::V ncmL, typename P2<R>::V cpR,
                                                      typename P2<R>::V A, typename P2<R>::V B,
                                                      typename P2<R>::V m1, typename P2<R>::V c,
                                                      typename P2<R>::V p1, typename P2<R>::V qm,
                                                      typename P2<R>::V qc, typename P2<R>::V qp, bool plm) {
  using P = P2<R>;
  if (!plm) return P::fma(ncmL, m1, P::fma(cpR, p1, P::mul(A, c)));
  return P::fma(ncmL, qm, P::fma(P::mk(-cpR.x, -cpR.y), qp, P::fma(B, qc, P::fma(ncmL, m1, P::fma(cpR, p1, P::mul(A, c))))));
}

// face_div with the optical-depth factors of Sec. 2.4: at a face with cells
// L | R the upwind state is multiplied by 1 - g_L + g = 1 + d (from L) or
// 1 - g_R + g = 1 - d (from R), d = f (1/n^0bar_L - 1/n^0bar_R) / 2; dlo and
// dhi are d of the lower (m1 | c) and upper (c | p1) faces.
template <typename R>
__device__ __forceinline__ typename P2<R>::V face_div_tau(unsigned um, unsigned up, typename P2<R>::V cm,
                                                        typename P2<R>::V cp, typename P2<R>::V m1,
                                                        typename P2<R>::V c, typename P2<R>::V p1,
                                                        typename P2<R>::V qm, typename P2<R>::V qc,
                                                        typename P2<R>::V qp, typename P2<R>::V dlo,
                                                        typename P2<R>::V dhi) {
  using P = P2<R>;
  const bool umx = um & 1, umy = um & 2, upx = up & 1, upy = up & 2;
  const auto one = P::mk(R(1), R(1));
  auto loR = P::mul(P::sub(c, qc), P::sub(one, dlo)), loL = P::mul(P::add(m1, qm), P::add(one, dlo));
  auto hiR = P::mul(P::sub(p1, qp), P::sub(one, dhi)), hiL = P::mul(P::add(c, qc), P::add(one, dhi));
  return P::sub(P::mul(cp, sel2<R>(upx, upy, hiR, hiL)), P::mul(cm, sel2<R>(umx, umy, loR, loL)));
}

// ---------------------------------------------------------------- TMA
// One-dimensional bulk copies (the TMA engine) global -> shared, completing
// on an mbarrier with a transaction count.  Rows are n_ap elements, a
// multiple of 16 bytes, and start on 16-byte boundaries.
constexpr int kMaxStages = 4;       // deepest ring of the stencil pipeline (the launcher picks 2 or 3)
constexpr int kStageMaxThreads = 512;   // consumers (two bins each) + one producer warp
// rows per ring stage: the x1 block (2h + 1 rows), the 2h x2 rows, the own
// row at k + h and the own row of I^0, with h = 2 (DC, PLM) or 3 (PPM)
__host__ __device__ constexpr int stage_rows(int recon) { return recon == RAD_RECON_PPM ? 15 : 11; }
constexpr long long kSpinLimit = 1ll << 28;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // a healthy wait takes microseconds

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s_addr(dst)),
      "l"(src), "r"(bytes), "r"(s_addr(bar))
      : "memory");
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the given phase parity of an mbarrier; false after limit_ns (or
// kSpinLimit polls), so that a wait that can no longer complete ends in an
// error status instead of a stalled kernel.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity,
                                                 unsigned long long limit_ns = kWaitLimitNs) {
  const uint32_t a = s_addr(bar);
  unsigned long long t0 = 0;
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 0) {
      const unsigned long long now = global_ns();
      if (it == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
  return false;
}

// Shared-memory footprint (bytes) of k_stage.
template <typename R, bool ANG>
__host__ __device__ constexpr size_t stage_smem(int threads, int nap, int kc, int depth, bool tau, int rows,
                                                bool mapr = false) {
  return (size_t)depth * rows * nap * sizeof(R)                 // staged stencil rows
         + (mapr ? (size_t)4 * nap * sizeof(R) : 0)             // MAPR gradients of two cells
         + (size_t)kc * nap * sizeof(R)                         // I* of the chunk
         + (size_t)kc * 8 * sizeof(R)                           // gas ux uy uz alphaE u0 (+3 pad: vector loads)
         + (size_t)kc * (threads / 32) * kNRedC * sizeof(R)     // per-warp partial sums
         + (size_t)kc * sizeof(R)                               // S per cell
         + (tau ? (size_t)kc * 6 * 5 * sizeof(R) : 0)           // optical-depth data of the six faces
         + (size_t)2 * kMaxStages * 8 + 16;                     // full and empty mbarriers
}

template <typename R, bool ANG, int RC, bool ST2, bool TAU, int AR = 0, int NAP = 0>
// AR: angular reconstruction, 0 donor cell, 1 PLM along the lines of a
// latitude-longitude grid, 2 minimum-angle planes (MAPR) on a geodesic grid.
// NAP: the padded row length when fixed at compile time (0: a.nap; < 0: -NAP,
// with the halo and frequency terms).
// Register budget: the flat FP32 DC / PLM kernels are held to 96 registers
// (the bound of a 544-thread block) so that five 128-thread CTAs fit an SM;
// the others get 128 (the curved kernels' CTAs are limited by shared memory
// first, and their angular-flux coefficients live in registers).
__global__ void __launch_bounds__((sizeof(R) == 4 && !ANG && RC != RAD_RECON_PPM) ? 544 : kStageMaxThreads) k_stage(StageArgs a) {
  using Col = typename GeoTypes<R>::Col;
  using Face = typename GeoTypes<R>::Face;
  using P = P2<R>;
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool AP = AR == 1, AM = AR == 2;
  // the kernels with a run-time row length also read halo rows of faces
  // shared with other blocks and add a multigroup frequency divergence; the
  // fixed-row variants (the common grids' fast path) compile without either
  // (a negative NAP is the fixed row length -NAP with both: the level-4
  // flat kernel of the block path)
  constexpr bool EXT = NAP <= 0;
  const int nap = NAP > 0 ? NAP : (NAP < 0 ? -NAP : a.nap);   // padded bins per row
  const int t = threadIdx.x;
  const int ncons = blockDim.x - 32;                      // consumer threads; the last warp produces
  const bool cons = t < ncons;
  const int nwarp = ncons >> 5;                           // consumer warps
  const int lane = t & 31, warp = t >> 5;
  const int b0 = 2 * t;                                   // bins b0, b0 + 1
  const bool inpair = b0 < nap;                         // pair inside the padded row
  const bool act0 = b0 < a.nang, act1 = b0 + 1 < a.nang;
  const int nchunk = (a.n3 + a.kc - 1) / a.kc;
  const int col = blockIdx.x / nchunk;
  const int chunk = blockIdx.x % nchunk;
  const int i = col % a.n1, j = col / a.n1;
  const int k0 = chunk * a.kc;
  const int nc = min(a.kc, a.n3 - k0);
  const unsigned ncol = (unsigned)a.n1 * a.n2;
  const unsigned strideK = ncol * (unsigned)nap;        // element offsets fit in 32 bits (host-checked)
  const R *Ip = (const R *)a.Iprev;
  const R *I0 = (const R *)a.I0;
  R *Io = (R *)a.Iout;
  constexpr bool plm = RC == RAD_RECON_PLM;
  constexpr bool ppm = RC == RAD_RECON_PPM;
  constexpr int H = ppm ? 3 : 2;                           // stencil half-width
  constexpr int X1N = 2 * H + 1, X2N = 2 * H;              // rows of the x1 block, x2 rows
  constexpr int SX2 = X1N, SX3 = X1N + X2N, SI0 = SX3 + 1, ROWS = SI0 + 1;   // ring slots
  const bool couple = a.mode != RAD_COUPLE_NONE;

  // shared memory: staged rows, I* of the chunk, then small per-cell arrays
  R *stg = (R *)smem_raw;                                  // [depth][ROWS][nap]
  R *sI = stg + a.depth * ROWS * nap;                    // [kc][nap]
  R *sgas = sI + a.kc * nap;                             // [kc][8]
  R *red = sgas + a.kc * 8;                                // [kc][nwarp][kNRedC]
  R *Sc = red + a.kc * nwarp * kNRedC;                     // [kc]
  constexpr bool tau = TAU;                                // optical-depth flux weighting (Sec. 2.4)
  R *stau = Sc + a.kc;                                     // [kc][6 faces][f, u^1, u^2, u^3, u^0 of the neighbour]
  R *gbuf = stau + (tau ? a.kc * 30 : 0);                 // [2][nap][2] MAPR gradients (two cells in turn)
  uint64_t *bars = (uint64_t *)(((uintptr_t)(gbuf + (AM ? 4 * nap : 0)) + 15) & ~(uintptr_t)15);   // [depth] full
  uint64_t *ebars = bars + kMaxStages;                                                // [depth] empty

  for (int c = t; c < nc; c += blockDim.x) {
    const unsigned cell = (unsigned)(k0 + c) * ncol + col;
    if (couple || tau) {
      const R ux = (R)a.u[3 * cell], uy = (R)a.u[3 * cell + 1], uz = (R)a.u[3 * cell + 2];
      sgas[8 * c + 0] = ux;
      sgas[8 * c + 1] = uy;
      sgas[8 * c + 2] = uz;
      sgas[8 * c + 3] = (R)a.aa[cell] + (R)a.as[cell];
      sgas[8 * c + 4] = sqrt(R(1) + ux * ux + uy * uy + uz * uz);
    }
  }
  if (tau) {
    // optical-depth weighting (Sec. 2.4): per cell and face, the face's
    // f = -expm1(-tau^2) with tau = C alpha_E dt / u^0hat from the face
    // averages of u and alpha_E, and the neighbour's velocity (for its n^0bar)
    for (int q = t; q < nc * 6; q += blockDim.x) {
      const int c = q / 6, s = q % 6, d = s >> 1, sg = (s & 1) ? 1 : -1;
      R *o = stau + (c * 6 + s) * 5;
      if (d >= a.ndim) {
        o[0] = R(0);
        o[1] = o[2] = o[3] = R(0);
        o[4] = R(1);
        continue;
      }
      const int k = k0 + c;
      int ii = i, jj = j, kk = k, pol = 0;
      if (d == 0) ii = wrap_idx<EXT>(i + sg, a.n1, a.bc_lo[0], a.bc_hi[0], pol);
      if (d == 1) {
        jj = wrap_idx<EXT>(j + sg, a.n2, a.bc_lo[1], a.bc_hi[1], pol);
        if (pol == 1 && a.n3 > 1) kk = (k + a.n3 / 2) % a.n3;
      }
      if (d == 2) kk = wrap_idx<EXT>(k + sg, a.n3, a.bc_lo[2], a.bc_hi[2], pol);
      const unsigned cell = (unsigned)k * ncol + col;
      const unsigned nbc = (unsigned)kk * ncol + (unsigned)jj * a.n1 + ii;
      const R uxo = (R)a.u[3 * cell], uyo = (R)a.u[3 * cell + 1], uzo = (R)a.u[3 * cell + 2];
      const R uxn = (R)a.u[3 * nbc], uyn = (R)a.u[3 * nbc + 1], uzn = (R)a.u[3 * nbc + 2];
      const R aEo = (R)a.aa[cell] + (R)a.as[cell], aEn = (R)a.aa[nbc] + (R)a.as[nbc];
      const R fx = R(0.5) * (uxo + uxn), fy = R(0.5) * (uyo + uyn), fz = R(0.5) * (uzo + uzn);
      const R u0F = sqrt(R(1) + fx * fx + fy * fy + fz * fz);
      const R tq = (R)a.tau_const * (R(0.5) * (aEo + aEn)) * (R)a.dt / u0F;
      o[0] = -rexpm1(-tq * tq);
      o[1] = uxn;
      o[2] = uyn;
      o[3] = uzn;
      o[4] = sqrt(R(1) + uxn * uxn + uyn * uyn + uzn * uzn);
    }
  }

  // ---- per-bin prefactors of this column (pair)
  const Col &cg = ((const Col *)a.cols)[col];
  R nx_[2] = {R(0), R(0)}, ny_[2] = {R(0), R(0)}, nz_[2] = {R(0), R(0)}, dO_[2] = {R(1), R(1)};
  for (int e = 0; e < 2; ++e) {
    if (b0 + e < a.nang) {
      nx_[e] = (R)a.dir[3 * (b0 + e)];
      ny_[e] = (R)a.dir[3 * (b0 + e) + 1];
      nz_[e] = (R)a.dir[3 * (b0 + e) + 2];
      dO_[e] = (R)a.dOmega[b0 + e];
    }
  }
  const V nhx = P::mk(nx_[0], nx_[1]), nhy = P::mk(ny_[0], ny_[1]), nhz = P::mk(nz_[0], nz_[1]);
  const V dOm = P::mk(act0 ? dO_[0] : R(0), act1 ? dO_[1] : R(0));
  const R n0up = cg.n0up;
  const V nlow0 = P::fma(nhz, P::mk(cg.M[0][3], cg.M[0][3]),
                         P::fma(nhy, P::mk(cg.M[0][2], cg.M[0][2]),
                                P::fma(nhx, P::mk(cg.M[0][1], cg.M[0][1]), P::mk(cg.M[0][0], cg.M[0][0]))));
  const V fconv = P::mul(P::mk(n0up, n0up), nlow0);                 // U = n^0 n_0 I
  const bool g0 = act0 && a.zero_guard && fabs((double)nlow0.x) < a.n0crit;
  const bool g1 = act1 && a.zero_guard && fabs((double)nlow0.y) < a.n0crit;
  // primitive recovery factor (0 for guarded or inactive bins)
  const V inv_f = P::mk((act0 && !g0) ? R(1) / fconv.x : R(0), (act1 && !g1) ? R(1) / fconv.y : R(0));
  const V keep = P::mk((act0 && !g0) ? R(1) : R(0), (act1 && !g1) ? R(1) : R(0));   // 0: guarded or padding
  // The stage combination of U = n^0 n_0 I, U* = U^{s-1} + dt L (stage 1) or
  // (U^0 + U^1 + dt L) / 2 (stage 2) with L = -(divS + divA), taken back to
  // I* = U* / (n^0 n_0) in one affine step (the FP64 kernels): I* = kS
  // (I^{s-1} [+ I^0]) + kD div with kS = 1 (1/2 in stage 2) and kD = -dt /
  // (n^0 n_0) (halved in stage 2); both 0 for guarded and padding bins.
  const R hs = ST2 ? R(0.5) : R(1);
  const V kS = P::mul(P::mk(hs, hs), keep);
  const V kD = P::mul(P::mk(-hs * (R)a.dt, -hs * (R)a.dt), inv_f);
  const R invdV = cg.invdV;
  auto fcoef = [&](const Face &F, unsigned &upR) -> V {
    V na = P::fma(nhz, P::mk(F.ea[3], F.ea[3]),
                  P::fma(nhy, P::mk(F.ea[2], F.ea[2]), P::fma(nhx, P::mk(F.ea[1], F.ea[1]), P::mk(F.ea[0], F.ea[0]))));
    V n0 = P::fma(nhz, P::mk(F.m0[3], F.m0[3]),
                  P::fma(nhy, P::mk(F.m0[2], F.m0[2]), P::fma(nhx, P::mk(F.m0[1], F.m0[1]), P::mk(F.m0[0], F.m0[0]))));
    upR = (na.x < R(0) ? 1u : 0u) | (na.y < R(0) ? 2u : 0u);
    V c = P::mul(P::mul(na, n0), P::mk(F.dA * invdV, F.dA * invdV));
    return P::mk(act0 ? c.x : R(0), act1 ? c.y : R(0));
  };
  V cm[3], cp[3];
  unsigned um[3] = {0u, 0u, 0u}, up[3] = {0u, 0u, 0u};
  for (int d = 0; d < 3; ++d) cm[d] = cp[d] = P::mk(R(0), R(0));
  {
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
  // weighted coefficients for the flat kernels (the curved ones keep the
  // select form: their registers go to the angular-flux coefficients)
  V ncmL[3], ncmR[3], cpL[3], cpR[3], gA[3], gB[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ncmR[d] = P::mk((um[d] & 1) ? -cm[d].x : R(0), (um[d] & 2) ? -cm[d].y : R(0));
    ncmL[d] = P::mk((um[d] & 1) ? R(0) : -cm[d].x, (um[d] & 2) ? R(0) : -cm[d].y);
    cpR[d] = P::mk((up[d] & 1) ? cp[d].x : R(0), (up[d] & 2) ? cp[d].y : R(0));
    cpL[d] = P::mk((up[d] & 1) ? R(0) : cp[d].x, (up[d] & 2) ? R(0) : cp[d].y);
    gA[d] = P::add(ncmR[d], cpL[d]);
    gB[d] = P::sub(cpL[d], ncmR[d]);
  }
  // Flat space without the optical-depth weighting, with the bins numbered
  // in sign pairs (a.sign_pairs; the fixed-row variants are launched only
  // then): along x1 and x2 both faces of a bin take their upwind states from
  // the same side, and both bins of a thread's pair from the same side too.
  // Mirrored so that the upwind neighbour u1 (and u2 beyond it) lies on the
  // left and the downwind neighbour d1 on the right,
  //   div = X (c + q(u1, c, d1)) + Y (u1 + q(u2, u1, c)),
  // X = cp, Y = -cm (upwind on the lower side) or X = -cm, Y = cp (upper),
  // with q the van Leer half-slope, odd under the mirror (so the mirrored
  // slopes carry their signs): two slopes and two coefficients per
  // dimension instead of three and four.  mo[d] holds the element offsets
  // of the rows u2, u1, d1 in a ring stage.
  constexpr bool MIR = !ANG && !TAU && RC != RAD_RECON_PPM;
  const bool mir = MIR && (NAP != 0 || a.sign_pairs);
  // In FP64 x3 takes the same form from the register window (its selects run
  // on the integer pipe, beside the FP64 pipe that bounds that kernel); mXs
  // is X with the sign of the mirror, which multiplies the own slope.
  constexpr bool MIR3 = MIR && sizeof(R) == 8;
  V mX[3], mY[3], mXs = P::mk(R(0), R(0));
  bool dn3 = false;
  int mo[2][3];
  if (MIR) {
#pragma unroll
    for (int d = 0; d < (MIR3 ? 3 : 2); ++d) {
      // the side of the element with the larger coefficient; a direction
      // component that is zero up to rounding (a few 1e-17: lattice points on
      // a coordinate plane) may carry either sign, and its flux is negligible
      // whichever side it takes
      const R ax = fabs(cm[d].x) + fabs(cp[d].x), ay = fabs(cm[d].y) + fabs(cp[d].y);
      const bool rx = um[d] & 1, ry = um[d] & 2;
      const bool dn = ax >= ay ? rx : ry;                // upwind on the upper side
      if (mir && rx != ry && fmin(ax, ay) > R(1e-6) * fmax(ax, ay)) atomicOr(a.err, kErrState);
      const V ncm = P::mk(-cm[d].x, -cm[d].y);
      mX[d] = dn ? ncm : cp[d];
      mY[d] = dn ? cp[d] : ncm;
      if (d == 2) {
        dn3 = dn;
        mXs = dn ? P::mk(-mX[2].x, -mX[2].y) : mX[2];
        continue;
      }
      // x1: the block rows i-2 .. i+2 in slots 0 .. 4; x2: rows j-2, j-1,
      // j+1, j+2 in slots SX2 .. SX2 + 3
      const int s2 = d == 0 ? (dn ? 4 : 0) : SX2 + (dn ? 3 : 0);
      const int s1 = d == 0 ? (dn ? 3 : 1) : SX2 + (dn ? 2 : 1);
      const int sd = d == 0 ? (dn ? 1 : 3) : SX2 + (dn ? 1 : 2);
      const int bo = inpair ? b0 : 0;
      mo[d][0] = s2 * nap + bo;
      mo[d][1] = s1 * nap + bo;
      mo[d][2] = sd * nap + bo;
    }
  }
  auto divm = [&](int d, const R *sr, V c) -> V {
    const V u1 = *(const V *)(sr + mo[d][1]);
    if (!plm) return P::fma(mX[d], c, P::mul(mY[d], u1));
    const V u2 = *(const V *)(sr + mo[d][0]), d1 = *(const V *)(sr + mo[d][2]);
    const V qf = vl2<R>(u2, u1, c), qc = vl2<R>(u1, c, d1);
    return P::fma(mX[d], P::add(c, qc), P::mul(mY[d], P::add(u1, qf)));
  };
  auto divd = [&](int d, V m1, V c, V p1, V qm, V qc, V qp, V dl, V dh) -> V {
    if (tau) return face_div_tau<R>(um[d], up[d], cm[d], cp[d], m1, c, p1, qm, qc, qp, dl, dh);
    if (ANG) return face_div<R>(um[d], up[d], cm[d], cp[d], m1, c, p1, qm, qc, qp);
    return face_div_g<R>(ncmL[d], cpR[d], gA[d], gB[d], m1, c, p1, qm, qc, qp, plm);
  };
  // the same from given face states (loL | loR at the lower face, hiL | hiR at the upper)
  auto divs = [&](int d, V loL, V loR, V hiL, V hiR, V dl, V dh) -> V {
    if (tau) {
      const V one = P::mk(R(1), R(1));
      loL = P::mul(loL, P::add(one, dl));
      loR = P::mul(loR, P::sub(one, dl));
      hiL = P::mul(hiL, P::add(one, dh));
      hiR = P::mul(hiR, P::sub(one, dh));
    }
    if (ANG || tau) {
      const bool umx = um[d] & 1, umy = um[d] & 2, upx = up[d] & 1, upy = up[d] & 2;
      return P::sub(P::mul(cp[d], sel2<R>(upx, upy, hiR, hiL)), P::mul(cm[d], sel2<R>(umx, umy, loR, loL)));
    }
    return P::fma(ncmR[d], loR, P::fma(ncmL[d], loL, P::fma(cpR[d], hiR, P::mul(cpL[d], hiL))));
  };
  // angular flux of each bin: divA = a_self I + sum_s a_nb[s] I_{m_s}
  R a_self[2] = {R(0), R(0)}, a_nb[2][kMaxSlots];
  R xu[2][kMaxSlots][2];      // MAPR: gnomonic coordinates of each side's midpoint in its upwind cell's plane
  int nb_m[2][kMaxSlots];
  if (ANG) {
    // unrolled in FP32 so that the coefficients stay in registers; the FP64
    // kernels keep them in local memory (they are bound by the FP64 pipe)
#pragma unroll(sizeof(R) == 4 ? 2 : 1)
    for (int e = 0; e < 2; ++e) {
      const int n = b0 + e;
      const bool ac = n < a.nang;
      R self = R(0);
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        a_nb[e][s] = R(0);
        nb_m[e][s] = ac ? n : 0;
        xu[e][s][0] = xu[e][s][1] = R(0);
        int m = ac ? a.slot_nbr[6 * n + s] : -1;
        if (m < 0) continue;
        nb_m[e][s] = m;
        int ed = a.slot_edge[6 * n + s];
        const double *eg = a.edge_geo + 8 * ed;
        R x = (R)eg[0], y = (R)eg[1], z = (R)eg[2], v0 = (R)eg[3], v1 = (R)eg[4], v2 = (R)eg[5], len = (R)eg[6];
        R pr[10] = {R(1), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
        R q0 = R(0), q1 = R(0), q2 = R(0);
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          q0 += cg.K[0][p] * pr[p];
          q1 += cg.K[1][p] * pr[p];
          q2 += cg.K[2][p] * pr[p];
        }
        R sp = -(v0 * q0 + v1 * q1 + v2 * q2);          // V . nu (nu is normal to n_e)
        R n0e = cg.M[0][0] + cg.M[0][1] * x + cg.M[0][2] * y + cg.M[0][3] * z;
        R Pv = len * sp * n0e;
        R PL = sp >= R(0) ? Pv : R(0), PR = sp >= R(0) ? R(0) : Pv;
        R dOn = e ? dO_[1] : dO_[0];
        const bool isp = a.edge_pq[2 * ed] == n;
        if (AP) {
          // the flux out of n through this side is cs times the upwind cell's
          // reconstruction at the side; kept: cs, and packed the neighbour m,
          // the cell of the upwind line beyond the side (behind n when n is
          // upwind, beyond m otherwise) and whether n is upwind
          const bool upn = isp ? sp >= R(0) : sp < R(0);
          const int *el = a.edge_line + 2 * ed;
          const int l = upn ? el[isp ? 0 : 1] : el[isp ? 1 : 0];
          a_nb[e][s] = (isp ? Pv : -Pv) / dOn;
          nb_m[e][s] = m | (l << 12) | (upn ? 1 << 24 : 0);
        } else if (AM) {
          // as above, with the upwind cell's plane evaluated at the side's
          // midpoint (its gnomonic coordinates in that cell's tangent plane)
          const bool upn = isp ? sp >= R(0) : sp < R(0);
          a_nb[e][s] = (isp ? Pv : -Pv) / dOn;
          nb_m[e][s] = m | (upn ? 1 << 24 : 0);
          const double *xs = (upn ? a.mapr_xo : a.mapr_xn) + 12 * n + 2 * s;
          xu[e][s][0] = (R)xs[0];
          xu[e][s][1] = (R)xs[1];
        } else if (isp) {
          self += PL;
          a_nb[e][s] = PR / dOn;
        } else {
          self -= PR;
          a_nb[e][s] = -PL / dOn;
        }
      }
      a_self[e] = ac ? self / (e ? dO_[1] : dO_[0]) : R(0);
    }
  }
  // ---- stencil rows of one cell (h = 2, or 3 for PPM): the contiguous x1
  // block (rows i-h..i+h, or one copy per row at a boundary), the 2h x2 rows,
  // this column's row at k+h (x3 window) and, in stage 2, this column's row
  // of I^0.  Slots: 0..2h x1 block (h = own), then the x2 rows j-h..j+h
  // without j, then own k+h, then I^0.
  // row kinds (wrap_idx): x1 rows 0 or a halo side (2, 3); x2 rows 0, the
  // polar mirror (1) or a halo side
  int xs[X1N], xk[X1N], yj[X2N], ypol[X2N];
  bool x1contig = true;
  for (int q = 0; q < X1N; ++q) {
    int kind = 0;
    xs[q] = q == H ? i : wrap_idx<EXT>(i + q - H, a.n1, a.bc_lo[0], a.bc_hi[0], kind);
    xk[q] = kind;
    if (xs[q] != i + q - H || (EXT && kind)) x1contig = false;
  }
  bool anypol = false;
  for (int q = 0; q < X2N; ++q) {
    int pol = 0;
    const int o = q < H ? q - H : q - H + 1;
    yj[q] = a.ndim >= 2 ? wrap_idx<EXT>(j + o, a.n2, a.bc_lo[1], a.bc_hi[1], pol) : j;
    ypol[q] = pol;
    anypol |= pol == 1;
  }
  const bool d3 = a.ndim >= 3;
  const size_t rowb = (size_t)nap * sizeof(R);
  auto rowp = [&](const R *base, int ii, int jj, int kk) {
    return base + ((size_t)kk * ncol + (size_t)jj * a.n1 + ii) * nap;
  };
  // this column's row at plane k (any k: wrapped, clamped or a halo row)
  auto kidx = [&](int k) {
    int kind;
    return wrap_idx<EXT>(k, a.n3, a.bc_lo[2], a.bc_hi[2], kind);
  };
  auto krow = [&](int k) -> const R * {
    int kind;
    const int kk = wrap_idx<EXT>(k, a.n3, a.bc_lo[2], a.bc_hi[2], kind);
    if (EXT && kind >= 2) return halo_row<R>(a.halo, a.n1, a.n2, a.n3, 2, kind - 2, kk, i, j, 0, nap);
    return rowp(Ip, i, j, kk);
  };
  auto produce = [&](int c, int st) {   // issue the copies of cell k0 + c into ring stage st
    const int k = k0 + c;
    R *dst = stg + (size_t)st * ROWS * nap;
    uint32_t bytes = (uint32_t)(X1N * rowb) + (a.ndim >= 2 ? (uint32_t)(X2N * rowb) : 0u) +
                     (d3 ? (uint32_t)rowb : 0u) + (ST2 ? (uint32_t)rowb : 0u);
    mbar_expect_tx(&bars[st], bytes);
    if (x1contig) {
      bulk_g2s(dst, rowp(Ip, i - H, j, k), (uint32_t)(X1N * rowb), &bars[st]);
    } else {
      for (int q = 0; q < X1N; ++q) {
        const R *src = (EXT && xk[q] >= 2) ? halo_row<R>(a.halo, a.n1, a.n2, a.n3, 0, xk[q] - 2, xs[q], 0, j, k, nap)
                                           : rowp(Ip, xs[q], j, k);
        bulk_g2s(dst + q * nap, src, (uint32_t)rowb, &bars[st]);
      }
    }
    if (a.ndim >= 2) {
      for (int q = 0; q < X2N; ++q) {
        const R *src;
        if (EXT && ypol[q] >= 2) {
          src = halo_row<R>(a.halo, a.n1, a.n2, a.n3, 1, ypol[q] - 2, yj[q], i, 0, k, nap);
        } else {
          int kk = k;
          if (ypol[q] == 1 && a.n3 > 1) kk = (k + a.n3 / 2) % a.n3;
          src = rowp(Ip, i, yj[q], kk);
        }
        bulk_g2s(dst + (SX2 + q) * nap, src, (uint32_t)rowb, &bars[st]);
      }
    }
    if (d3) bulk_g2s(dst + SX3 * nap, EXT ? krow(k + H) : rowp(Ip, i, j, kidx(k + H)), (uint32_t)rowb, &bars[st]);
    if (ST2) bulk_g2s(dst + SI0 * nap, rowp(I0, i, j, k), (uint32_t)rowb, &bars[st]);
  };
  const int p0 = act0 ? a.perm[b0] : 0, p1 = act1 ? a.perm[b0 + 1] : 0;
  const unsigned own = (unsigned)col * nap + (inpair ? b0 : 0);
  const int bb = inpair ? b0 : 0;
  auto sv = [&](const R *row) -> V { return *(const V *)(row + bb); };
  const R dtR = (R)a.dt, dts = (R)a.dts;
  const R c2pre = dts / R(kFourPi);
  const V zero = P::mk(R(0), R(0));
  if (t == 0) {
    for (int st = 0; st < a.depth; ++st) {
      mbar_init(&bars[st], 1);
      mbar_init(&ebars[st], (uint32_t)nwarp);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();   // gas staged, barriers initialised
  bool timeout = false;
  if (!cons) {
    // ---- producer warp: one lane issues every cell's copies into the ring,
    // waiting for the consumers to release a stage before refilling it
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;                      // parity of the empty barrier's next phase
      for (int c = 0; c < nc; ++c) {
        if (c >= a.depth && !mbar_wait_parity(&ebars[st], ph)) {
          timeout = true;     // the consumers time out on the full barrier in turn
          break;
        }
        produce(c, st);
        if (++st == a.depth) {
          st = 0;
          if (c >= a.depth) ph ^= 1u;
        }
      }
    }
  }

  // ---- phase A (consumer warps): transport, stage combination, primitive I*, coupling sums
  V w0 = zero, w1 = zero, w2 = zero, w3 = zero, qa = zero, qb = zero;   // x3 window and slopes
  V pw[6];                                               // PPM x3 window, rows k-3 .. k+2
#pragma unroll
  for (int q = 0; q < 6; ++q) pw[q] = zero;
  if (ppm && cons && d3) {
#pragma unroll
    for (int q = 0; q < 6; ++q)
      pw[q] = EXT ? __ldg((const V *)(krow(k0 - 3 + q) + bb))
                  : __ldg((const V *)(Ip + (unsigned)kidx(k0 - 3 + q) * strideK + own));
  }
  if (!ppm && cons && d3) {
    if (EXT) {
      w0 = __ldg((const V *)(krow(k0 - 2) + bb));
      w1 = __ldg((const V *)(krow(k0 - 1) + bb));
      w2 = __ldg((const V *)(krow(k0) + bb));
      w3 = __ldg((const V *)(krow(k0 + 1) + bb));
    } else {
      w0 = __ldg((const V *)(Ip + (unsigned)kidx(k0 - 2) * strideK + own));
      w1 = __ldg((const V *)(Ip + (unsigned)kidx(k0 - 1) * strideK + own));
      w2 = __ldg((const V *)(Ip + (unsigned)kidx(k0) * strideK + own));
      w3 = __ldg((const V *)(Ip + (unsigned)kidx(k0 + 1) * strideK + own));
    }
    if (plm) {
      qa = vl2<R>(w0, w1, w2);
      qb = vl2<R>(w1, w2, w3);
    }
  }
  int st = 0;
  uint32_t ph = 0;                          // parity of the full barrier's current phase
  for (int c = 0; c < (cons ? nc : 0); ++c) {
    const R *sr = stg + (size_t)st * ROWS * nap;
    if (!mbar_wait_parity(&bars[st], ph)) timeout = true;
    V zc, sx = zero;
    // optical-depth factors d of the six faces (zero without the weighting)
    V dlo[3] = {zero, zero, zero}, dhi[3] = {zero, zero, zero};
    if (tau) {
      const GasRow<R> grow = gas_load(sgas + 8 * c);
      const R *g = grow.v;
      const V io = P::rcp(P::sub(P::mk(g[4], g[4]), P::fma(P::mk(g[2], g[2]), nhz,
                                 P::fma(P::mk(g[1], g[1]), nhy, P::mul(P::mk(g[0], g[0]), nhx)))));
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) break;
        const R *tl = stau + (c * 6 + 2 * d) * 5, *th = tl + 5;
        const V im = P::rcp(P::sub(P::mk(tl[4], tl[4]), P::fma(P::mk(tl[3], tl[3]), nhz,
                                   P::fma(P::mk(tl[2], tl[2]), nhy, P::mul(P::mk(tl[1], tl[1]), nhx)))));
        const V ip = P::rcp(P::sub(P::mk(th[4], th[4]), P::fma(P::mk(th[3], th[3]), nhz,
                                   P::fma(P::mk(th[2], th[2]), nhy, P::mul(P::mk(th[1], th[1]), nhx)))));
        dlo[d] = P::mul(P::mk(R(0.5) * tl[0], R(0.5) * tl[0]), P::sub(im, io));
        dhi[d] = P::mul(P::mk(R(0.5) * th[0], R(0.5) * th[0]), P::sub(io, ip));
      }
    }
    if (d3 && ppm) {
      V win[7];
#pragma unroll
      for (int q = 0; q < 6; ++q) win[q] = pw[q];
      win[6] = sv(sr + SX3 * nap);
      zc = win[3];
      V loL, loR, hiL, hiR;
      ppm_states<R>(win, loL, loR, hiL, hiR);
      sx = divs(2, loL, loR, hiL, hiR, dlo[2], dhi[2]);
#pragma unroll
      for (int q = 0; q < 6; ++q) pw[q] = win[q + 1];
    } else if (d3) {
      const V w4 = sv(sr + SX3 * nap);
      const V qc = plm ? vl2<R>(w2, w3, w4) : zero;   // slope of k+1
      zc = w2;
      // slopes: qa = slope(k-1), qb = slope(k), qc = slope(k+1)
      if (MIR3 && mir) {
        // upwind frame: u1 = w1 or w3, its mirrored slope qa or -qc, the
        // own mirrored slope +-qb (the sign in mXs)
        const V u1 = dn3 ? w3 : w1;
        sx = plm ? P::fma(mX[2], w2, P::fma(mXs, qb, P::mul(mY[2], P::add(u1, dn3 ? P::mk(-qc.x, -qc.y) : qa))))
                 : P::fma(mX[2], w2, P::mul(mY[2], u1));
      } else {
        sx = divd(2, w1, w2, w3, qa, qb, qc, dlo[2], dhi[2]);
      }
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = w4;
      qa = qb;
      qb = qc;
    } else {
      zc = sv(sr + H * nap);
    }
    if (ppm) {
      V v[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) v[q] = q == H ? zc : sv(sr + q * nap);
      V loL, loR, hiL, hiR;
      ppm_states<R>(v, loL, loR, hiL, hiR);
      sx = P::add(sx, divs(0, loL, loR, hiL, hiR, dlo[0], dhi[0]));
    } else if (mir) {
      sx = P::add(sx, divm(0, sr, zc));
    } else {
      const V m2 = sv(sr), m1 = sv(sr + nap), q1 = sv(sr + 3 * nap), q2 = sv(sr + 4 * nap);
      V sm = zero, sc = zero, sp = zero;
      if (plm) {
        sm = vl2<R>(m2, m1, zc);
        sc = vl2<R>(m1, zc, q1);
        sp = vl2<R>(zc, q1, q2);
      }
      sx = P::add(sx, divd(0, m1, zc, q1, sm, sc, sp, dlo[0], dhi[0]));
    }
    if (a.ndim >= 2 && ppm) {
      V v[7];
      v[H] = zc;
#pragma unroll
      for (int q = 0; q < X2N; ++q) {
        const R *row = sr + (SX2 + q) * nap;
        v[q < H ? q : q + 1] = (ANG && anypol && ypol[q] == 1) ? P::mk(row[p0], row[p1]) : sv(row);
      }
      V loL, loR, hiL, hiR;
      ppm_states<R>(v, loL, loR, hiL, hiR);
      sx = P::add(sx, divs(1, loL, loR, hiL, hiR, dlo[1], dhi[1]));
    } else if (a.ndim >= 2 && mir) {
      sx = P::add(sx, divm(1, sr, zc));
    } else if (a.ndim >= 2) {
      V yv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const R *row = sr + (SX2 + q) * nap;
        yv[q] = (ANG && anypol && ypol[q] == 1) ? P::mk(row[p0], row[p1]) : sv(row);
      }
      V sm = zero, sc = zero, sp = zero;
      if (plm) {
        sm = vl2<R>(yv[0], yv[1], zc);
        sc = vl2<R>(yv[1], zc, yv[2]);
        sp = vl2<R>(zc, yv[2], yv[3]);
      }
      sx = P::add(sx, divd(1, yv[1], zc, yv[2], sm, sc, sp, dlo[1], dhi[1]));
    }
    V divA = zero;
    if (ANG && AM) {
      // minimum-angle planes (MAPR): each bin's flattest plane through itself
      // and two cyclically adjacent neighbours (gradient g = inv (dI_a, dI_b)),
      // shared through shared memory (two cells' buffers in turn, so one
      // barrier of the consumer warps per cell suffices), then every side's
      // flux from its upwind cell's plane at the side's midpoint
      const R *row = sr + H * nap;
      R *gb = gbuf + (c & 1) * 2 * nap;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = b0 + e;
        if (n < a.nang) {
          const R In = e ? zc.y : zc.x;
          const int *nbc = a.mapr_nb + 6 * n;
          const double *mi = a.mapr_minv + 24 * n;
          R dl[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const int m = nbc[q];
            dl[q] = m >= 0 ? row[m] - In : R(0);
          }
          const int K = nbc[5] >= 0 ? 6 : 5;
          R gx = R(0), gy = R(0), bq = R(0);
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            if (q < K) {
              const int q2 = q + 1 == K ? 0 : q + 1;
              const R x = (R)mi[4 * q] * dl[q] + (R)mi[4 * q + 1] * dl[q2];
              const R y = (R)mi[4 * q + 2] * dl[q] + (R)mi[4 * q + 3] * dl[q2];
              const R qq = x * x + y * y;
              if (q == 0 || qq < bq) {
                bq = qq;
                gx = x;
                gy = y;
              }
            }
          }
          gb[2 * n] = gx;
          gb[2 * n + 1] = gy;
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(ncons) : "memory");
      R da[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = b0 + e;
        R acc = R(0);
#pragma unroll
        for (int s2 = 0; s2 < kMaxSlots; ++s2) {
          const int pk = nb_m[e][s2];
          const int u = (pk >> 24) & 1 ? n : (pk & 0xfff);
          acc += a_nb[e][s2] * (row[u] + gb[2 * u] * xu[e][s2][0] + gb[2 * u + 1] * xu[e][s2][1]);
        }
        da[e] = acc;
      }
      divA = P::mk(da[0], da[1]);
    } else if (ANG) {
      // the own row of this cell is slot h of the staged x1 block
      const R *row = sr + H * nap;
      R da[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const R In = e ? zc.y : zc.x;
        R acc = a_self[e] * In;
#pragma unroll
        for (int s2 = 0; s2 < kMaxSlots; ++s2) {
          if (AP) {
            // PLM along the grid line: y + q(x, y, z) is the reconstruction of
            // the upwind cell y at the side towards z, x the cell behind y
            const int pk = nb_m[e][s2];
            const R Im = row[pk & 0xfff], Il = row[(pk >> 12) & 0xfff];
            const bool upn = (pk >> 24) & 1;
            const R y = upn ? In : Im, z = upn ? Im : In;
            acc += a_nb[e][s2] * (y + vl_half(Il, y, z));
          } else {
            acc += a_nb[e][s2] * row[nb_m[e][s2]];
          }
        }
        da[e] = acc;
      }
      divA = P::mk(da[0], da[1]);
    }
    // U* = U^{s-1} + dt L   (stage 1)   or   U^0/2 + (U^1 + dt L)/2   (stage 2), L = -(divS + divA)
    if (ANG) sx = P::add(sx, divA);
    if (EXT && a.divF) sx = P::add(sx, __ldg((const V *)((const R *)a.divF + (unsigned)(k0 + c) * strideK + own)));
    // FP64: the affine form (fewer FP64-pipe operations); FP32: U* first and
    // I* after the release (the FP32 kernels' register allocation prefers it)
    constexpr bool AFF = sizeof(R) == 8;
    V Is = zero, Us = zero;
    if (AFF) {
      Is = ST2 ? P::fma(kS, P::add(sv(sr + SI0 * nap), zc), P::mul(kD, sx)) : P::fma(kS, zc, P::mul(kD, sx));
    } else {
      Us = P::fma(P::mk(-dtR, -dtR), sx, P::mul(fconv, zc));   // L = -(divS + divA)
      if (ST2) {
        const V U0 = P::mul(fconv, sv(sr + SI0 * nap));
        Us = P::mul(P::mk(R(0.5), R(0.5)), P::add(U0, Us));
      }
    }
    // every read of this ring stage is done: release it to the producer now,
    // so that the next copies overlap this cell's coupling sums (the
    // arrive's release semantics order the warp's reads before it)
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&ebars[st])) : "memory");
    }
    if (!AFF) Is = P::mul(Us, inv_f);
    if (inpair) *(V *)(sI + c * nap + b0) = Is;
    if (a.Istar && inpair) *(V *)((R *)a.Istar + (unsigned)(k0 + c) * strideK + own) = Is;
    if (couple) {
      const GasRow<R> grow = gas_load(sgas + 8 * c);
      const R *g = grow.v;
      const V ux = P::mk(g[0], g[0]), uy = P::mk(g[1], g[1]), uz = P::mk(g[2], g[2]);
      const R aEd = g[3] * dts;
      const V nb = P::sub(P::mk(g[4], g[4]), P::fma(uz, nhz, P::fma(uy, nhy, P::mul(ux, nhx))));
      const V nbaE = P::mul(nb, P::mk(aEd, aEd));
      // r2 = 1 / (n^0bar den), den = n^0 + n^0bar alpha_E dt: one reciprocal
      // gives both 1 / den = n^0bar r2 and dOmega / (n^0bar den)
      const V r2 = P::rcp(P::mul(nb, P::add(P::mk(n0up, n0up), nbaE)));
      const V w = P::mul(P::mul(Is, P::mul(nb, nb)), dOm);                 // Ibar dOmega_bar
      const V v0 = P::mul(P::mul(P::mk(-nbaE.x, -nbaE.y), P::mul(nb, r2)), w);   // (c1 - 1) Ibar dOmega_bar
      const V v1 = P::mul(dOm, r2);                                          // dOmega / (n^0bar den)
      const R s2 = warp_reduce4(v0.x + v0.y, v1.x + v1.y, w.x + w.y, R(0), lane);
      if ((lane & 7) == 0 && lane < 24) red[(c * nwarp + warp) * kNRedC + (lane >> 3)] = s2;
    }
    if (++st == a.depth) {
      st = 0;
      ph ^= 1u;
    }
  }
  if (timeout) atomicOr(a.err, 1 << 3);

  double psrc[4] = {0.0, 0.0, 0.0, 0.0};
  if (couple) {
    __syncthreads();
    // ---- phase B: one thread per cell; its gas loads are issued before it
    // sums the warps' partials, so that their latency overlaps the sums
    if (t < nc) {
      const int c = t, k = k0 + c;
      const unsigned cell = (unsigned)k * ncol + col;
      if (ST2 && a.src) {                  // stage 1's share of the source, added to in phase D
#pragma unroll
        for (int m = 0; m < 4; ++m) psrc[m] = a.src[4 * cell + m];
      }
      const double Tst = ST2 ? 0.5 * (a.T0[cell] + a.T1[cell]) : a.T0[cell];
      const double aa = a.aa[cell], as = a.as[cell];
      R rs[kNRedA] = {R(0), R(0), R(0)};
      for (int w = 0; w < nwarp; ++w)
#pragma unroll
        for (int r = 0; r < kNRedA; ++r) rs[r] += red[(c * nwarp + w) * kNRedC + r];
      const double D = (double)rs[0], A2 = a.dts / kFourPi * (double)rs[1], Em = (double)rs[2];
      double S, Tp = Tst;
      bool ok = true;
      if (a.mode == RAD_COUPLE_THERMAL) {
        const double cv = a.rho[cell] * a.inv_gm1;
        const double B4 = A2 * aa * a.a_rad;
        const double B1 = cv * (1.0 - A2 * as);
        const double B0 = D + A2 * as * Em - B1 * Tst;   // A1 - B1 T- - (1 - A2 alpha_s) Ebar-
        Tp = quartic_root(B4, B1, B0, sizeof(R) == 8, ok, Tst);
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
  } else {
    __syncthreads();
    if (t < nc) {
      const unsigned cell = (unsigned)(k0 + t) * ncol + col;
      a.Tout[cell] = ST2 ? 0.5 * (a.T0[cell] + a.T1[cell]) : a.T0[cell];
      if (a.src && !ST2) {
        for (int m = 0; m < 4; ++m) a.src[4 * cell + m] = 0.0;
      }
    }
  }

  // ---- phase C: implicit update of every bin
  V chk = zero;           // stays 0 unless a written value is not finite (0 * inf, 0 * nan = nan)
  const bool want_src = couple && a.src;
  // I+ of one cell before the guard, from I* and the cell's source S
  auto implicit = [&](int c, V &Is, V &out) {
    Is = inpair ? *(const V *)(sI + c * nap + b0) : zero;
    out = Is;
    if (couple) {
      const GasRow<R> grow = gas_load(sgas + 8 * c);
      const R *g = grow.v;
      const V ux = P::mk(g[0], g[0]), uy = P::mk(g[1], g[1]), uz = P::mk(g[2], g[2]);
      const R aEd = g[3] * dts;
      const V nb = P::sub(P::mk(g[4], g[4]), P::fma(uz, nhz, P::fma(uy, nhy, P::mul(ux, nhx))));
      // q = 1 / (den n^0bar^3): c2 / n^0bar^3 = c2pre q and n^0 / den = n^0 n^0bar^3 q
      const V nb3 = P::mul(nb, P::mul(nb, nb));
      const V q = P::rcp(P::mul(P::fma(nb, P::mk(aEd, aEd), P::mk(n0up, n0up)), nb3));
      const V c2n = P::mul(P::mk(c2pre, c2pre), q);
      out = P::fma(P::mul(P::mul(P::mk(n0up, n0up), nb3), q), Is, P::mul(c2n, P::mk(Sc[c], Sc[c])));
    }
  };
  // gas source: the pair's share of sum (I+ - I*) n^A dOmega (before the guard)
  auto src4 = [&](V Is, V out, R (&v)[4]) {
    const V d = P::mul(P::sub(out, Is), dOm);
    const V dx = P::mul(d, nhx), dy = P::mul(d, nhy), dz = P::mul(d, nhz);
    v[0] = d.x + d.y;
    v[1] = dx.x + dx.y;
    v[2] = dy.x + dy.y;
    v[3] = dz.x + dz.y;
  };
  auto store = [&](int c, V out) {
    out = P::mul(out, keep);
    if (inpair) {
      *(V *)(Io + (unsigned)(k0 + c) * strideK + own) = out;
      chk = P::fma(out, zero, chk);
    }
  };
  // cells in fours, then pairs: the cells' source sums share one
  // reduce-scatter and their arithmetic interleaves
  int c = 0;
  for (; c + 7 < (cons ? nc : 0); c += 8) {
    V Is[8], out[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) implicit(c + e, Is[e], out[e]);
    if (want_src) {
      R v[32];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        R ve[4];
        src4(Is[e], out[e], ve);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[4 * e + q] = ve[q];
      }
      const R s = warp_reduce32<R>(v, lane);
      red[((c + (lane >> 2)) * nwarp + warp) * kNRedC + (lane & 3)] = s;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) store(c + e, out[e]);
  }
  for (; c + 3 < (cons ? nc : 0); c += 4) {
    V Is[4], out[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) implicit(c + e, Is[e], out[e]);
    if (want_src) {
      R v[16];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        R ve[4];
        src4(Is[e], out[e], ve);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[4 * e + q] = ve[q];
      }
      const R s = warp_reduce16<R>(v, lane);
      if ((lane & 1) == 0) {
        const int q = lane >> 1;
        red[((c + (q >> 2)) * nwarp + warp) * kNRedC + (q & 3)] = s;
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) store(c + e, out[e]);
  }
  for (; c + 1 < (cons ? nc : 0); c += 2) {
    V Isa, outa, Isb, outb;
    implicit(c, Isa, outa);
    implicit(c + 1, Isb, outb);
    if (want_src) {
      R v[8], va[4], vb[4];
      src4(Isa, outa, va);
      src4(Isb, outb, vb);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = va[q];
        v[4 + q] = vb[q];
      }
      const R s = warp_reduce8<R>(v, lane);
      if ((lane & 3) == 0) {
        const int q = lane >> 2;
        red[((c + (q >> 2)) * nwarp + warp) * kNRedC + (q & 3)] = s;
      }
    }
    store(c, outa);
    store(c + 1, outb);
  }
  if (cons && c < nc) {
    V Is, out;
    implicit(c, Is, out);
    if (want_src) {
      R v[4];
      src4(Is, out, v);
      const R s = warp_reduce4(v[0], v[1], v[2], v[3], lane);
      if ((lane & 7) == 0) red[(c * nwarp + warp) * kNRedC + (lane >> 3)] = s;
    }
    store(c, out);
  }
  const bool bad = !isfinite(chk.x) || !isfinite(chk.y);
  if (cons && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonFinite);
  if (want_src) {
    // ---- phase D: -dR^0_mu with dR^0_mu = n^0 M[mu][A] sum (I+ - I*) n^A dOmega
    __syncthreads();
    if (t < nc) {
      const int c = t;
      const unsigned cell = (unsigned)(k0 + c) * ncol + col;
      R xs[4];
#pragma unroll
      for (int A = 0; A < 4; ++A) {
        R s = R(0);
        for (int w = 0; w < nwarp; ++w) s += red[(c * nwarp + w) * kNRedC + A];
        xs[A] = s;
      }
      double *sp = a.src + 4 * cell;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        R dR = n0up * (cg.M[m][0] * xs[0] + cg.M[m][1] * xs[1] + cg.M[m][2] * xs[2] + cg.M[m][3] * xs[3]);
        sp[m] = ST2 ? psrc[m] - (double)dR : -0.5 * (double)dR;
      }
    }
  }
}

}  // namespace rad
