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
//                      DC / PLM / PPM upwind stencil and of the angular
//                      fluxes; adjoint_kernels.cuh, adjoint_tadj_*.cu)
// with (a, b, beta) = (0, 1, 1) for stage 1 and (1/2, 1/2, 1/2) for stage 2.
// With the optical-depth weighting of Sec. 2.4 every face's lambda weight
// carries the face's factor (1 +- d), and the factor's dependence on
// alpha_E = alpha_a + alpha_s (through f = -expm1(-tau^2)) gives a further
// opacity gradient: each cell reduces over bins the flux derivative of its
// lower face in each dimension (k_transport_adj), and k_tau_grad adds the
// two faces on either side of a cell to dL/dalpha_a and dL/dalpha_s.
// The PLM and PPM limiters are differentiated on their active branches.
// Boundary conditions enter through the transpose of the neighbour map:
// periodic wrap and outflow clamp by matching every stencil position's
// source cell against the target (a face that appears twice in the window
// of a short periodic line counts once), the polar map by explicit terms
// for the faces next to a pole whose upwind stencils reach across it (the
// pole faces themselves have zero area).  No atomics: every output element
// is written by one thread.
#include "adjoint_kernels.cuh"

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
      // with the radiation-dominated substitution the velocity is itself a
      // function of the intensities: dL/du through every n^0bar = u^0 - u.n
      double dudn[3] = {0.0, 0.0, 0.0};
      if (A.lam_u && act) {
        const double inb = 1.0 / nbd;
        const double drden = -(aad + asd) * dtsd * rdend * rdend;
        const double dLdnb = lrden * drden - 3.0 * c2pd * rdend * inb * inb * inb * inb * S * lpd +
                             (cm1d * Isd * lD + Isd * lEm) * 2.0 * nbd * dOd - lA2s * dOd * rdend * inb * inb;
        const double u0d = sqrt(1.0 + uxd * uxd + uyd * uyd + uzd * uzd);
        dudn[0] = dLdnb * (uxd / u0d - xh);
        dudn[1] = dLdnb * (uyd / u0d - yh);
        dudn[2] = dLdnb * (uzd / u0d - zh);
      }
      double t2[4];
      cta_sum4<double>(act ? -nbd * dtsd * rdend * rdend * lrden : 0.0, dudn[0], dudn[1], dudn[2], dbuf, nwarp,
                       lane, warp, t2);
      if (n == 0 && A.lam_u) {
        A.lam_u[3 * cell] = t2[1];
        A.lam_u[3 * cell + 1] = t2[2];
        A.lam_u[3 * cell + 2] = t2[3];
      }
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

namespace {

template <typename R>
cudaError_t launch_transport_adj_any(const AdjArgs &A, bool ang, cudaStream_t st) {
  if (ang && A.s.recon_ang == RAD_RECON_PLM) return launch_transport_adj<R, true, 1>(A, st);
  if (ang && A.s.recon_ang == RAD_RECON_MAPR) return launch_transport_adj<R, true, 2>(A, st);
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
  const size_t need = 5 * ib + 12 * tb;
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
  double *usub = (double *)(p + 5 * ib + 6 * tb);    // [cell][3] substituted velocity (rad_dom)
  double *lamu = (double *)(p + 5 * ib + 9 * tb);    // [cell][3] dL/du of the substituted velocity (rad_dom)
  const bool rd = o->rad_dom != 0;
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
  // with the radiation-dominated substitution the forward stage is the
  // transport-only stage kernel followed by the substituted coupling
  if (rd) s.mode = RAD_COUPLE_NONE;
  cudaError_t ce = launch_stage(s, f32, ang, ctx->stream);
  if (ce == cudaSuccess && rd) ce = launch_couple_rd(s, f32, T1, T1, ctx->stream);
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
  s.mode = o->coupling;
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
  A.lam_u = nullptr;
  // the coupling adjoint of one stage; with rad_dom the coupling ran at the
  // substituted velocity: recompute it, take the coupling back at it (which
  // also gives dL/du), then take dL/du back through the substitution
  auto couple_adj = [&](const void *Istar, const double *Tm) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (rd) {
      e = launch_rd_sub(0, A.s, f32, Istar, Tm, usub, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                        0.0, ctx->stream);
      A.s.u = usub;
      A.lam_u = lamu;
    }
    if (e == cudaSuccess) e = f32 ? launch_couple_adj<float>(A, ctx->stream) : launch_couple_adj<double>(A, ctx->stream);
    if (rd) {
      A.s.u = gas->u;
      A.lam_u = nullptr;
      if (e == cudaSuccess)
        e = launch_rd_sub(1, A.s, f32, Istar, Tm, nullptr, lamu, A.mu, g_aa, g_as, A.outTa, A.wTa, A.outTb, A.wTb,
                          ctx->stream);
    }
    return e;
  };
  if (ce == cudaSuccess) {
    A.s.dts = 0.5 * dt;
    A.s.stage2 = 1;
    A.lam = lam_np1;
    A.Istar = I2s;
    A.mu = mu;
    ce = couple_adj(I2s, T2);     // T2 holds the stage's T- = (T^0 + T^1) / 2
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
    ce = couple_adj(I1s, gas->T);
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
