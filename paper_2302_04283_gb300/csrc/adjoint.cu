// Reverse-mode step (hand-written adjoint) and the outgoing-flux loss.
//
// rad_step_adjoint recomputes the two stages of rad_step from the checkpoint
// I_n (keeping I^1 and both pre-coupling primitives I^1*, I^2*) and then
// runs the stages backwards:
//   coupling adjoint   lambda_I+  ->  mu = lambda_U* = lambda_I* / (n^0 n_0),
//                      and dL/d(alpha_a, alpha_s, eta) of this coupling
//                      (k_couple_adj: per-cell reductions, as in the forward);
//                      with thermal coupling also lambda_T+ -> lambda_T-,
//                      through the root of the quartic by the implicit-function
//                      theorem (dT+ = -(T^4 dB4 + T dB1 + dB0) / f'(T+))
//   transport adjoint  mu -> lambda_{I^{s-1}} += b f mu + b beta dt J_L^T mu,
//                      lambda_{I^0} += a f mu
//                      (k_transport_adj: gather form of the transposed
//                      PLM / DC upwind stencil and of the angular fluxes)
// with (a, b, beta) = (0, 1, 1) for stage 1 and (1/2, 1/2, 1/2) for stage 2.
// With the optical-depth weighting of Sec. 2.4 every face's lambda weight
// carries the face's factor (1 +- d), and the factor's dependence on
// alpha_E = alpha_a + alpha_s (through f = -expm1(-tau^2)) gives a further
// opacity gradient: each cell reduces over bins the flux derivative of its
// lower face in each dimension (k_transport_adj), and k_tau_grad adds the
// two faces on either side of a cell to dL/dalpha_a and dL/dalpha_s.
// The PLM limiter is differentiated on its active branch.  Boundary
// conditions enter through the transpose of the neighbour map: periodic
// wrap and outflow clamp by matching every stencil position's source cell
// against the target, the polar map by one explicit term (the only polar
// face whose stencil reaches a ghost with non-zero area is the first /
// last interior face).  No atomics: every output element is written by one
// thread.
#include "step_kernel.cuh"

namespace rad {

// L = sum_{k,j} sum_{n: n^1 > 0 at the outer x1 face} I[k][j][n1-1][n] dOmega_n.
// One block per (j, k) row; the outer-face tetrad row gives the sign of n^1.
template <typename R>
__global__ void k_loss(const R *I, R *dL, double *L, int n1, int n2, int nap, int nang, const FaceGeo *f1,
                       const double *dir, const double *dOmega) {
  int row = blockIdx.x;            // k * n2 + j
  int j = row % n2;
  const FaceGeo &F = f1[j * (n1 + 1) + n1];
  long long base = ((long long)row * n1 + (n1 - 1)) * nap;
  double acc = 0.0;
  for (int n = threadIdx.x; n < nang; n += blockDim.x) {
    double na = F.ea[0] + F.ea[1] * dir[3 * n] + F.ea[2] * dir[3 * n + 1] + F.ea[3] * dir[3 * n + 2];
    double w = na > 0.0 ? dOmega[n] : 0.0;
    acc += w * (double)I[base + n];
    if (dL) dL[base + n] = (R)w;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    L[row] = s;                      // per-row partial; summed in order below
  }
}

// Fixed-order sum of the row partials (deterministic loss).
__global__ void k_sum_rows(const double *part, int rows, double *L) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += part[r];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *L = sh[0];
}

int launch_loss(rad_ctx *ctx, const void *I, int precision, double *L, void *dL, std::string &err) {
  const DevGeom &G = ctx->geom;
  size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  size_t esz = precision == RAD_F32 ? 4 : 8;
  if (dL) cudaMemsetAsync(dL, 0, ncell * ctx->ang.n_ap * esz, ctx->stream);
  unsigned rows = (unsigned)(G.n[1] * G.n[2]);
  if (ctx->loss_rows < (int)rows) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->loss_buf);
    ctx->loss_buf = nullptr;
    ctx->loss_rows = 0;
    if (cudaMalloc(&ctx->loss_buf, rows * sizeof(double)) != cudaSuccess) {
      err = "loss scratch allocation failed";
      return RAD_ENOMEM;
    }
    ctx->loss_rows = (int)rows;
  }
  if (precision == RAD_F32)
    k_loss<float><<<rows, 256, 0, ctx->stream>>>((const float *)I, (float *)dL, ctx->loss_buf, G.n[0], G.n[1],
                                                 ctx->ang.n_ap, ctx->ang.n_ang, G.f1, ctx->dang.dir,
                                                 ctx->dang.dOmega);
  else
    k_loss<double><<<rows, 256, 0, ctx->stream>>>((const double *)I, (double *)dL, ctx->loss_buf, G.n[0], G.n[1],
                                                  ctx->ang.n_ap, ctx->ang.n_ang, G.f1, ctx->dang.dir,
                                                  ctx->dang.dOmega);
  k_sum_rows<<<1, 256, 0, ctx->stream>>>(ctx->loss_buf, (int)rows, L);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("loss launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

// ---------------------------------------------------------------- adjoint
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

// Adjoint of the coupling of one stage (thermal, fixed emissivity or none).
template <typename R, int MAXT>
__global__ void __launch_bounds__(MAXT) k_couple_adj(AdjArgs A) {
  using Col = typename GeoTypes<R>::Col;
  const StageArgs &a = A.s;
  __shared__ R buf[32 * 4];
  __shared__ double dbuf[32 * 4], sc[8];
  const int n = threadIdx.x;
  const int nwarp = blockDim.x >> 5, lane = n & 31, warp = n >> 5;
  const bool act = n < a.nang;
  const int nchunk = (a.n3 + a.kc - 1) / a.kc;
  const int col = blockIdx.x / nchunk, chunk = blockIdx.x % nchunk;
  const int k0 = chunk * a.kc, nc = min(a.kc, a.n3 - k0);
  const long long ncol = (long long)a.n1 * a.n2;
  const long long strideK = ncol * a.nap;
  const long long own = (long long)col * a.nap + (act ? n : 0);
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
  const R fconv = n0up * nlow0;
  const bool guard = act && a.zero_guard && fabs((double)nlow0) < a.n0crit;
  const R inv_f = act ? R(1) / fconv : R(0);
  const R dts = (R)a.dts, c2pre = dts / R(kFourPi);
  const R *lam = (const R *)A.lam, *Isv = (const R *)A.Istar;
  R *mu = (R *)A.mu;
  for (int c = 0; c < nc; ++c) {
    const int k = k0 + c;
    const long long cell = (long long)k * ncol + col;
    const long long e = (long long)k * strideK + own;
    const R lamp = (act && !guard) ? lam[e] : R(0);
    if (a.mode == RAD_COUPLE_NONE) {
      if (act) mu[e] = guard ? R(0) : lamp * inv_f;
      continue;
    }
    const R ux = (R)a.u[3 * cell], uy = (R)a.u[3 * cell + 1], uz = (R)a.u[3 * cell + 2];
    const R aE = (R)(a.aa[cell] + a.as[cell]), as = (R)a.as[cell];
    const R u0 = sqrt(R(1) + ux * ux + uy * uy + uz * uz);
    const R Is = act ? Isv[e] : R(0);
    const R nb = u0 - (ux * nh0 + uy * nh1 + uz * nh2);
    const R rden = R(1) / (n0up + nb * aE * dts);
    const R c1 = n0up * rden;
    const R c2n = c2pre * rden / (nb * nb * nb);
    const R wbar = nb * nb * dOm;
    if (a.mode == RAD_COUPLE_THERMAL) {
      // forward (Sec. 2.5): D = sum (c1 - 1) I* wbar, A2 = c2pre sum dOmega
      // rden / n^0bar, Ebar- = sum I* wbar, the quartic B4 T^4 + B1 T + B0 = 0,
      // Ebar+ = Ebar- - c_v (T+ - T-), S = alpha_a a T+^4 + alpha_s Ebar+,
      // I+ = c1 I* + c2n S.  The reverse sweep runs in FP64 for both
      // precisions (only I* and lambda_I+ are in the working precision): the
      // terms of dL/dalpha_s cancel, and FP32 per-bin sums lose percents.
      const ColGeo &cd = A.cols64[col];
      double xh = 0.0, yh = 0.0, zh = 0.0, dOd = 0.0;
      if (act) {
        xh = a.dir[3 * n];
        yh = a.dir[3 * n + 1];
        zh = a.dir[3 * n + 2];
        dOd = a.dOmega[n];
      }
      const double n0d = cd.n0up, dtsd = a.dts, c2pd = dtsd / kFourPi;
      const double uxd = a.u[3 * cell], uyd = a.u[3 * cell + 1], uzd = a.u[3 * cell + 2];
      const double aad = a.aa[cell], asd = a.as[cell], ar = a.a_rad;
      const double nbd = sqrt(1.0 + uxd * uxd + uyd * uyd + uzd * uzd) - (uxd * xh + uyd * yh + uzd * zh);
      const double nbaEd = nbd * (aad + asd) * dtsd;
      const double rdend = 1.0 / (n0d + nbaEd);
      const double c1d = n0d * rdend, cm1d = -nbaEd * rdend;          // c1 and c1 - 1
      const double c2nd = c2pd * rdend / (nbd * nbd * nbd);
      const double wbd = nbd * nbd * dOd;
      const double Isd = act ? (double)Is : 0.0, lpd = (double)lamp;
      double t4[4];
      cta_sum4<double>(act ? cm1d * Isd * wbd : 0.0, act ? dOd * rdend / nbd : 0.0, act ? Isd * wbd : 0.0,
                       act ? c2nd * lpd : 0.0, dbuf, nwarp, lane, warp, t4);
      if (n == 0) {
        const double D = t4[0], A2 = c2pd * t4[1], Em = t4[2], lS = t4[3];
        const double Tm = a.stage2 ? 0.5 * (a.T0[cell] + a.T1[cell]) : a.T0[cell];
        const double cv = a.rho[cell] * a.inv_gm1;
        const double B4 = A2 * aad * ar, B1 = cv * (1.0 - A2 * asd), B0 = D + A2 * asd * Em - B1 * Tm;
        bool ok = true;
        const double Tp = quartic_root(B4, B1, B0, true, ok);
        if (!ok || !isfinite(Tp)) atomicOr(a.err, kErrNoConv);
        const double T3 = Tp * Tp * Tp, T4 = T3 * Tp;
        const double Ep = Em - cv * (Tp - Tm);
        // S = alpha_a a T+^4 + alpha_s Ebar+
        double lT = (A.lamTp ? A.lamTp[cell] : 0.0) + 4.0 * aad * ar * T3 * lS;
        const double lEp = asd * lS;
        double laa = ar * T4 * lS, las = Ep * lS;
        // Ebar+ = Ebar- - c_v T+ + c_v T-
        double lEm = lEp, lTm = cv * lEp;
        lT -= cv * lEp;
        // T+ = root(B4, B1, B0): d/dB = -(T^4, T, 1) / f'(T+)
        const double g = lT / (4.0 * B4 * T3 + B1);
        const double lB4 = -g * T4, lB0 = -g;
        double lB1 = -g * Tp;
        // B0 = D + A2 alpha_s Ebar- - B1 T-
        double lA2 = asd * Em * lB0;
        las += A2 * Em * lB0;
        lEm += A2 * asd * lB0;
        lB1 -= Tm * lB0;
        lTm -= B1 * lB0;
        // B1 = c_v (1 - A2 alpha_s), B4 = A2 alpha_a a
        lA2 += -cv * asd * lB1 + aad * ar * lB4;
        las -= cv * A2 * lB1;
        laa += A2 * ar * lB4;
        sc[0] = aad * ar * T4 + asd * Ep;      // S
        sc[1] = lB0;                           // lambda_D
        sc[2] = lEm;
        sc[3] = c2pd * lA2;                    // lambda of sum dOmega rden / n^0bar
        sc[4] = laa;
        sc[5] = las;
        sc[6] = lTm;
      }
      __syncthreads();
      const double S = sc[0], lD = sc[1], lEm = sc[2], lA2s = sc[3];
      const double lc1 = Isd * lpd + Isd * wbd * lD;
      const double lIs = c1d * lpd + cm1d * wbd * lD + wbd * lEm;
      const double lrden = n0d * lc1 + c2pd / (nbd * nbd * nbd) * S * lpd + dOd / nbd * lA2s;
      double t2[4];
      cta_sum4<double>(act ? -nbd * dtsd * rdend * rdend * lrden : 0.0, 0.0, 0.0, 0.0, dbuf, nwarp, lane, warp, t2);
      if (n == 0) {
        const double laE = t2[0];
        A.g_aa[cell] += sc[4] + laE;
        A.g_as[cell] += sc[5] + laE;
        if (A.outTa) A.outTa[cell] = (A.accTa ? A.outTa[cell] : 0.0) + A.wTa * sc[6];
        if (A.outTb) A.outTb[cell] = A.wTb * sc[6];
      }
      if (act) {
        const double fd = n0d * (cd.M[0][0] + cd.M[0][1] * xh + cd.M[0][2] * yh + cd.M[0][3] * zh);
        mu[e] = guard ? R(0) : (R)(lIs / fd);
      }
      continue;
    }
    const R eta = (R)a.eta[cell];
    R t[3];
    cta_sum3<R>(act ? c1 * Is * wbar : R(0), act ? dOm * rden / nb : R(0), act ? c2n * lamp : R(0), buf, nwarp,
                lane, warp, t);
    const R A1 = t[0], A2 = c2pre * t[1], lS = t[2];
    const R Q = R(1) - A2 * as;
    const R Ep = (A1 + R(kFourPi) * A2 * eta) / Q;
    const R S = R(kFourPi) * eta + as * Ep;
    const R lEp = as * lS;
    const R lA1 = lEp / Q;
    const R lQ = -Ep * lEp / Q;
    const R lA2 = R(kFourPi) * eta * lEp / Q - as * lQ;
    const R leta = R(kFourPi) * lS + R(kFourPi) * A2 * lEp / Q;
    const R las = Ep * lS - A2 * lQ;
    const R lc1 = Is * lamp + Is * wbar * lA1;
    const R lc2n = S * lamp;
    const R lIs = c1 * lamp + c1 * wbar * lA1;
    const R lden = -c1 * rden * lc1 - c2n * rden * lc2n - c2pre * dOm * rden * rden / nb * lA2;
    R t2[3];
    cta_sum3<R>(act ? nb * dts * lden : R(0), R(0), R(0), buf, nwarp, lane, warp, t2);
    if (n == 0) {
      A.g_aa[cell] += (double)t2[0];
      A.g_as[cell] += (double)(t2[0] + las);
      if (A.g_eta) A.g_eta[cell] += (double)leta;
    }
    if (act) mu[e] = guard ? R(0) : lIs * inv_f;
  }
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

// Transposed transport of one stage (gather form, one thread per target bin).
template <typename R, bool ANG, int MAXT, bool TAU>
__global__ void __launch_bounds__(MAXT) k_transport_adj(AdjArgs A) {
  using Col = typename GeoTypes<R>::Col;
  using Face = typename GeoTypes<R>::Face;
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

  // per dimension: the 4 faces between positions (cr, cr+1), cr = -2..1, and
  // 1/dV at positions -2..2 (0 for ghosts of non-periodic dimensions)
  int nd = a.ndim;
  R cA[3][4], ivd[3][5];
  bool uR[3][4], fex[3][4];
  int N[3] = {a.n1, a.n2, a.n3};
  int y[3] = {i, j, 0};
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 4; ++t) {
      cA[d][t] = R(0);
      uR[d][t] = false;
      fex[d][t] = false;
    }
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 5; ++t) ivd[d][t] = R(0);
  for (int d = 0; d < nd && d < 2; ++d) {
    const bool per = a.bc_lo[d] == RAD_BC_PERIODIC;
    for (int t = 0; t < 5; ++t) {
      int p = y[d] + t - 2;
      bool ghost = p < 0 || p >= N[d];
      if (ghost && !per) continue;
      int pp = ((p % N[d]) + N[d]) % N[d];
      int c2 = d == 0 ? j * a.n1 + pp : pp * a.n1 + i;
      ivd[d][t] = cols[c2].invdV;
    }
    for (int t = 0; t < 4; ++t) {
      int c = y[d] + t - 2;          // face between cells c and c+1, face index c+1
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
    for (int t = 0; t < 4; ++t) {
      cA[2][t] = c3;
      uR[2][t] = act ? u : false;
    }
    for (int t = 0; t < 5; ++t) ivd[2][t] = cg.invdV;
  }
  // angular: transposed coefficients
  R at_self = R(0), at_nb[kMaxSlots];
  int nb_m[kMaxSlots];
  if (ANG) {
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
  // positions are handled separately)
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
      // stencil values at positions -3..3 and mu at -2..2 along d
      R v[7], m5[5];
      bool match[7];
      for (int t = 0; t < 7; ++t) {
        bool ghost, pol;
        int p = y[d] + t - 3;
        int q = src_idx(d, p, ghost, pol);
        int ii = i, jj = j, kk = k, bin = nb_self;
        if (d == 0) ii = q;
        if (d == 1) jj = q;
        if (d == 2) kk = q;
        if (pol) {
          kk = a.n3 > 1 ? (k + a.n3 / 2) % a.n3 : k;
          bin = nperm;
        }
        v[t] = act ? Il[addr(ii, jj, kk, bin)] : R(0);
        match[t] = !pol && (q == y[d]);
        if (t >= 1 && t <= 5) m5[t - 1] = (ghost && a.bc_lo[d] != RAD_BC_PERIODIC) || !act ? R(0)
                                                                                         : mu[addr(ii, jj, kk, bin)];
      }
      // optical-depth weighting: 1 / n^0bar of the cells at positions -2..2
      // and, per face t (positions t - 2 | t - 1), d_t and df/d(alpha_E)
      R nbi[5], fdt[4], dfa[4];
      if (tauw) {
        R ux5[5], uy5[5], uz5[5], ae5[5];
        for (int t = 0; t < 5; ++t) {
          bool ghost, pol;
          const int q = src_idx(d, y[d] + t - 2, ghost, pol);
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
        for (int t = 0; t < 4; ++t) {
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
      for (int t = 0; t < 4; ++t) {
        if (d == 2) {   // x3 faces exist unless they lie beyond a non-periodic boundary
          const int cf = k + t - 2;
          fex[2][t] = act && (a.bc_lo[2] == RAD_BC_PERIODIC || (cf >= -1 && cf <= a.n3 - 1));
        }
        if (!fex[d][t]) continue;
        // face between positions cr = t - 2 and cr + 1 (window index t + 1, t + 2)
        R lphi = -cA[d][t] * ivd[d][t] * m5[t] + cA[d][t] * ivd[d][t + 1] * m5[t + 1];
        const bool right = uR[d][t];
        const int s0 = right ? t + 1 : t;          // window index of the stencil's first cell
        if (tauw) {
          if (t == 1) {   // this cell's lower face: the flux's derivative in f
            const R ph = right ? v[3] - (plm ? half_slope(v[2], v[3], v[4]) : R(0))
                               : v[2] + (plm ? half_slope(v[1], v[2], v[3]) : R(0));
            gt[d] = lphi * ph * (right ? R(-0.5) : R(0.5)) * (nbi[1] - nbi[2]) * dfa[1];
          }
          lphi *= right ? R(1) - fdt[t] : R(1) + fdt[t];
        }
        R dd[3];
        dphi(plm, right, v[s0], v[s0 + 1], v[s0 + 2], dd);
        R g = R(0);
        for (int u = 0; u < 3; ++u)
          if (match[s0 + u]) g += dd[u];
        lam += lphi * g;
      }
    }
    // polar: the first / last interior x2 face reaches the ghost across the pole
    if (nd >= 2 && act && ((j == 0 && a.bc_lo[1] == RAD_BC_POLAR) || (j == a.n2 - 1 && a.bc_hi[1] == RAD_BC_POLAR))) {
      const bool lo = j == 0;
      const int kk = a.n3 > 1 ? (k + a.n3 / 2) % a.n3 : k;
      const int bp = nperm;                         // bin of the mirrored direction
      const R px = (R)a.dir[3 * bp], py = (R)a.dir[3 * bp + 1], pz = (R)a.dir[3 * bp + 2];
      const int fi = lo ? 1 : a.n2 - 1;             // face between rows fi-1 and fi
      bool u;
      const R cAf = face_coefA(F2[fi * a.n1 + i], px, py, pz, u);
      const bool needed = lo ? !u : u;              // stencil reaching row -1 (or n2)
      if (needed) {
        const int jl = fi - 1, jr = fi;
        R lphi = -cAf * cols[jl * a.n1 + i].invdV * mu[addr(i, jl, kk, bp)] +
                 cAf * cols[jr * a.n1 + i].invdV * mu[addr(i, jr, kk, bp)];
        if (tauw) {   // the factor of this face for bin bp (upwind side: the left cell for lo)
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
          lphi *= lo ? R(1) + df : R(1) - df;
        }
        R dd[3];
        if (lo) {   // stencil (-1, 0, 1) of the left cell 0; position -1 is this cell
          dphi(plm, false, Il[eown], Il[addr(i, 0, kk, bp)], Il[addr(i, 1, kk, bp)], dd);
          lam += lphi * dd[0];
        } else {    // stencil (n2-2, n2-1, n2) of the right cell; position n2 is this cell
          dphi(plm, true, Il[addr(i, a.n2 - 2, kk, bp)], Il[addr(i, a.n2 - 1, kk, bp)], Il[eown], dd);
          lam += lphi * dd[2];
        }
      }
    }
    if (ANG) {
      R ga = at_self * mu0;
      for (int s = 0; s < kMaxSlots; ++s) ga += at_nb[s] * mu[addr(i, j, k, nb_m[s])];
      lam -= ga;
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

namespace {

template <typename R, bool ANG>
cudaError_t launch_transport_adj(const AdjArgs &A, cudaStream_t st) {
  int threads = (A.s.nap + 31) / 32 * 32;
  int nchunk = (A.s.n3 + A.s.kc - 1) / A.s.kc;
  dim3 grid((unsigned)((long long)A.s.n1 * A.s.n2 * nchunk));
  const bool tau = A.s.tau_const > 0.0;
  if (threads <= 256)
    tau ? k_transport_adj<R, ANG, 256, true><<<grid, threads, 0, st>>>(A)
        : k_transport_adj<R, ANG, 256, false><<<grid, threads, 0, st>>>(A);
  else if (threads <= 512)
    tau ? k_transport_adj<R, ANG, 512, true><<<grid, threads, 0, st>>>(A)
        : k_transport_adj<R, ANG, 512, false><<<grid, threads, 0, st>>>(A);
  else
    tau ? k_transport_adj<R, ANG, 1024, true><<<grid, threads, 0, st>>>(A)
        : k_transport_adj<R, ANG, 1024, false><<<grid, threads, 0, st>>>(A);
  if (tau) {
    const StageArgs &a = A.s;
    const long long ncell = (long long)a.n1 * a.n2 * a.n3;
    k_tau_grad<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(
        A.gtau, a.n1, a.n2, a.n3, a.ndim, a.bc_lo[0] == RAD_BC_PERIODIC, a.bc_lo[1] == RAD_BC_PERIODIC,
        a.bc_lo[2] == RAD_BC_PERIODIC, A.wAL, A.g_aa, A.g_as);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_transport_adj_any(const AdjArgs &A, bool ang, cudaStream_t st) {
  return ang ? launch_transport_adj<R, true>(A, st) : launch_transport_adj<R, false>(A, st);
}

template <typename R>
cudaError_t launch_couple_adj(const AdjArgs &A, cudaStream_t st) {
  int threads = (A.s.nap + 31) / 32 * 32;
  int nchunk = (A.s.n3 + A.s.kc - 1) / A.s.kc;
  dim3 grid((unsigned)((long long)A.s.n1 * A.s.n2 * nchunk));
  if (threads <= 256) k_couple_adj<R, 256><<<grid, threads, 0, st>>>(A);
  else if (threads <= 512) k_couple_adj<R, 512><<<grid, threads, 0, st>>>(A);
  else k_couple_adj<R, 1024><<<grid, threads, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace

int launch_adjoint(rad_ctx *ctx, const void *I_n, const rad_gas *gas, double dt, const rad_opts *o,
                   const void *lam_np1, void *lam_n, const double *lamT_np1, double *lamT_n, double *g_aa,
                   double *g_as, double *g_eta, std::string &err) {
  const DevGeom &G = ctx->geom;
  const bool f32 = o->precision == RAD_F32;
  const bool ang = G.kind != RAD_MINK_CART;
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  const size_t esz = f32 ? 4 : 8;
  const size_t ib = (ncell * ctx->ang.n_ap * esz + 255) / 256 * 256;
  const size_t tb = (ncell * sizeof(double) + 255) / 256 * 256;
  const size_t need = 5 * ib + 6 * tb;
  if (ctx->adj_bytes < need) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->adj_buf);
    ctx->adj_buf = nullptr;
    ctx->adj_bytes = 0;
    if (cudaMalloc(&ctx->adj_buf, need) != cudaSuccess) {
      err = "adjoint scratch allocation failed";
      return RAD_ENOMEM;
    }
    ctx->adj_bytes = need;
  }
  unsigned char *p = (unsigned char *)ctx->adj_buf;
  void *I1 = p, *I1s = p + ib, *I2s = p + 2 * ib, *mu = p + 3 * ib, *lamI1 = p + 4 * ib;
  double *T1 = (double *)(p + 5 * ib), *T2 = (double *)(p + 5 * ib + tb);
  double *lamT1 = (double *)(p + 5 * ib + 2 * tb);   // adjoint of the stage-1 temperature
  double *gtau = (double *)(p + 5 * ib + 3 * tb);    // [cell][3] lower-face sums (optical-depth weighting)
  const bool thermal = o->coupling == RAD_COUPLE_THERMAL;
  if (!thermal && lamT_n && lamT_n != lamT_np1) {
    // the temperature passes through an uncoupled or fixed-emissivity step
    const cudaError_t te = lamT_np1 ? cudaMemcpyAsync(lamT_n, lamT_np1, ncell * sizeof(double),
                                                      cudaMemcpyDeviceToDevice, ctx->stream)
                                    : cudaMemsetAsync(lamT_n, 0, ncell * sizeof(double), ctx->stream);
    if (te != cudaSuccess) {
      err = std::string("adjoint temperature copy failed: ") + cudaGetErrorString(te);
      return RAD_ECUDA;
    }
  }
  // ---- forward recompute with the pre-coupling primitives kept
  StageArgs s = make_stage_args(ctx, gas, dt, o, nullptr);
  {
    const int rc = check_stage(s, f32, err);
    if (rc != RAD_OK) return rc;
  }
  s.Iprev = I_n;
  s.I0 = I_n;
  s.Iout = I1;
  s.Istar = I1s;
  s.T0 = gas->T;
  s.T1 = nullptr;
  s.Tout = T1;
  s.stage2 = 0;
  s.dts = dt;
  cudaError_t ce = launch_stage(s, f32, ang, ctx->stream);
  if (ce == cudaSuccess) {
    s.Iprev = I1;
    s.I0 = I_n;
    s.Iout = lamI1;     // stage-2 output is not needed; lamI1 is overwritten below
    s.Istar = I2s;
    s.T0 = gas->T;
    s.T1 = T1;
    s.Tout = T2;
    s.stage2 = 1;
    s.dts = 0.5 * dt;
    ce = launch_stage(s, f32, ang, ctx->stream);
  }
  s.Istar = nullptr;
  // ---- stage 2 backwards
  AdjArgs A;
  A.s = s;
  A.g_aa = g_aa;
  A.g_as = g_as;
  A.g_eta = g_eta;
  A.cols64 = G.cols;
  A.gtau = gtau;
  // temperature adjoint (thermal coupling): stage 2 takes lambda_T of the
  // step's output, T- = (T^0 + T^1) / 2 splits its lambda_T- in halves to
  // T^0 (lamT_n) and T^1 (lamT1); stage 1 takes lamT1 and adds its
  // lambda_T- (T- = T^0) to lamT_n
  A.lamTp = lamT_np1;
  A.outTa = lamT_n;
  A.wTa = 0.5;
  A.accTa = 0;
  A.outTb = lamT1;
  A.wTb = 0.5;
  if (ce == cudaSuccess) {
    A.s.dts = 0.5 * dt;
    A.s.stage2 = 1;
    A.lam = lam_np1;
    A.Istar = I2s;
    A.mu = mu;
    ce = f32 ? launch_couple_adj<float>(A, ctx->stream) : launch_couple_adj<double>(A, ctx->stream);
  }
  if (ce == cudaSuccess) {
    A.Ilin = I1;
    A.outA = lamI1;
    A.wAf = 0.5;
    A.wAL = 0.5 * dt;
    A.accA = 0;
    A.outB = lam_n;
    A.wBf = 0.5;
    A.accB = 0;
    ce = f32 ? launch_transport_adj_any<float>(A, ang, ctx->stream) : launch_transport_adj_any<double>(A, ang, ctx->stream);
  }
  // ---- stage 1 backwards
  if (ce == cudaSuccess) {
    A.s.dts = dt;
    A.s.stage2 = 0;
    A.lamTp = lamT1;
    A.outTa = lamT_n;
    A.wTa = 1.0;
    A.accTa = 1;
    A.outTb = nullptr;
    A.lam = lamI1;
    A.Istar = I1s;
    A.mu = mu;
    ce = f32 ? launch_couple_adj<float>(A, ctx->stream) : launch_couple_adj<double>(A, ctx->stream);
  }
  if (ce == cudaSuccess) {
    A.Ilin = I_n;
    A.outA = lam_n;
    A.wAf = 1.0;
    A.wAL = dt;
    A.accA = 1;
    A.outB = nullptr;
    ce = f32 ? launch_transport_adj_any<float>(A, ang, ctx->stream) : launch_transport_adj_any<double>(A, ang, ctx->stream);
  }
  if (ce != cudaSuccess) {
    err = std::string("adjoint launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
