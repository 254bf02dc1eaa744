// Host launchers of the stage kernel (two stages per SSP-RK2 step) and of
// the time-step bound.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "step_kernel.cuh"

namespace rad {

namespace {

// dt bound of one (column, bin); atomically reduced as the bit pattern of a
// positive double (order preserving).
__global__ void k_cfl(const ColGeo *cols, int n1, int n2, int ndim, const double *xf1, const double *xf2,
                      double dx3, int nang, const double *dir, const double *dOmega, const int *slot_nbr,
                      const int *slot_edge, const double *edge_geo, int ang, const double *edges, int ngroup,
                      unsigned long long *out) {
  int col = blockIdx.x;
  int n = threadIdx.x;
  if (n >= nang) return;
  int i = col % n1, j = col / n1;
  const ColGeo &cg = cols[col];
  double nh[4] = {1.0, dir[3 * n], dir[3 * n + 1], dir[3 * n + 2]};
  double best = INFINITY;
  double dx[3] = {xf1[i + 1] - xf1[i], xf2[j + 1] - xf2[j], dx3};
  double n0 = cg.n0up;
  for (int d = 0; d < ndim; ++d) {
    double na = 0.0;
    for (int A = 0; A < 4; ++A) na += cg.e[d + 1][A] * nh[A];
    double sp = fabs(na / n0);
    if (sp > 0.0) best = fmin(best, dx[d] / sp);
  }
  if (ang) {
    double rate = 0.0;
    for (int s = 0; s < kMaxSlots; ++s) {
      if (slot_nbr[6 * n + s] < 0) continue;
      const double *eg = edge_geo + 8 * slot_edge[6 * n + s];
      double x = eg[0], y = eg[1], z = eg[2];
      double pr[10] = {1.0, x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
      double q[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < 3; ++c)
        for (int p = 0; p < 10; ++p) q[c] += cg.K[c][p] * pr[p];
      double sp = -(eg[3] * q[0] + eg[4] * q[1] + eg[5] * q[2]);
      rate += eg[6] * fabs(sp);
    }
    if (rate > 0.0) best = fmin(best, dOmega[n] * n0 / rate);
  }
  if (ngroup > 0) {
    // multigroup: a group's donor-cell outflow through its upper edge must
    // not empty it within the step (n^0 dnu / (nu_hi |s|))
    const double pr[10] = {1.0, nh[1], nh[2], nh[3], nh[1] * nh[1], nh[1] * nh[2], nh[1] * nh[3],
                           nh[2] * nh[2], nh[2] * nh[3], nh[3] * nh[3]};
    double q0 = 0.0;
    for (int p = 0; p < 10; ++p) q0 += cg.K0[p] * pr[p];
    const double s = fabs(q0);
    for (int g = 0; g < ngroup && s > 0.0; ++g) {
      const double lo = edges[g], hi = edges[g + 1];
      if (isinf(hi)) continue;
      best = fmin(best, n0 * (hi - lo) / (hi * s));
    }
  }
  if (best < INFINITY) atomicMin(out, (unsigned long long)__double_as_longlong(best));
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// ever arrives at; the wait gives up after limit_ns and the error bit of a
// timed-out wait is set, exactly as in the stage and moment kernels.
__global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0 && !mbar_wait_parity(&bar, 0, limit_ns)) atomicOr(err, 1 << 3);
}

}  // namespace

cudaError_t launch_wait_selftest(rad_ctx *ctx, double seconds) {
  k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->err_word, (unsigned long long)(seconds * 1e9));
  return cudaGetLastError();
}

cudaError_t launch_stage(const StageArgs &a, bool f32, bool ang, cudaStream_t st) {
  bool ext = a.divF != nullptr;             // halo rows or a frequency divergence: the run-time-row kernels
  for (int f = 0; f < 6; ++f) ext |= a.halo[f] != nullptr;
  if (ext && !(ang && a.recon_ang != RAD_RECON_DC)) {
    if (f32 && !ang && a.nap == kNapGeo4 && a.sign_pairs) return launch_stage_rp<float, false, 0, -kNapGeo4>(a, st);
    if (f32) return ang ? launch_stage_rp<float, true>(a, st) : launch_stage_rp<float, false>(a, st);
    return ang ? launch_stage_rp<double, true>(a, st) : launch_stage_rp<double, false>(a, st);
  }
  if (ang && a.recon_ang == RAD_RECON_PLM)
    return f32 ? launch_stage_rp<float, true, 1>(a, st) : launch_stage_rp<double, true, 1>(a, st);
  if (ang && a.recon_ang == RAD_RECON_MAPR)
    return f32 ? launch_stage_rp<float, true, 2>(a, st) : launch_stage_rp<double, true, 2>(a, st);
  if (f32 && !ang && a.nap == kNapGeo4 && a.sign_pairs) return launch_stage_rp<float, false, 0, kNapGeo4>(a, st);
  if (f32 && ang) {
    if (a.nap == kNapGeo4) return launch_stage_rp<float, true, 0, kNapGeo4>(a, st);
    if (a.nap == kNapGeo6) return launch_stage_rp<float, true, 0, kNapGeo6>(a, st);
    if (a.nap == kNapGeo8) return launch_stage_rp<float, true, 0, kNapGeo8>(a, st);
  }
  if (f32) return ang ? launch_stage_rp<float, true>(a, st) : launch_stage_rp<float, false>(a, st);
  return ang ? launch_stage_rp<double, true>(a, st) : launch_stage_rp<double, false>(a, st);
}

StageArgs make_stage_args(rad_ctx *ctx, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src) {
  const DevGeom &G = ctx->geom;
  StageArgs a;
  a.Istar = nullptr;
  a.rho = gas->rho;
  a.u = gas->u;
  a.aa = gas->alpha_a;
  a.as = gas->alpha_s;
  a.eta = gas->eta;
  a.src = gas_src;
  a.dt = dt;
  a.dts = dt;
  a.stage2 = 0;
  a.n1 = G.n[0];
  a.n2 = G.n[1];
  a.n3 = G.n[2];
  a.nap = ctx->ang.n_ap;
  a.nang = ctx->ang.n_ang;
  a.sign_pairs = ctx->ang.sign_pairs ? 1 : 0;
  a.ndim = G.ndim;
  // ring depth and cells per CTA along x3: a 3-stage ring (2 when the bins
  // are too many for a chunk of min(n3, 8) cells within the shared-memory
  // budget), then the longest chunk (up to kMaxChunk) that fits.  Three
  // stages cover the copy latency and keep the 162-bin FP32 CTA small
  // enough for five per SM.
  {
    const int threads = (a.nap / 2 + 31) / 32 * 32;
    const bool f32 = o->precision == RAD_F32;
    auto smem = [&](int kc, int depth) {
      const bool mapr = o->recon_ang == RAD_RECON_MAPR;
      return f32 ? stage_smem<float, false>(threads, a.nap, kc, depth, o->tau_const > 0.0, stage_rows(o->recon), mapr)
                 : stage_smem<double, false>(threads, a.nap, kc, depth, o->tau_const > 0.0, stage_rows(o->recon), mapr);
    };
    const size_t budget = (size_t)200 * 1024;
    const int kmax = G.ndim >= 3 ? std::min(G.n[2], kMaxChunk) : 1;
    const int kwant = std::min(kmax, 8);
    int depth = 3;
    while (depth > 2 && smem(kwant, depth) > budget) --depth;
    int kc = kmax;
    while (kc > 1 && smem(kc, depth) > budget) --kc;
    a.depth = depth;
    a.kc = kc;
  }
  for (int d = 0; d < 3; ++d) {
    a.bc_lo[d] = G.bc_lo[d];
    a.bc_hi[d] = G.bc_hi[d];
  }
  const bool f32 = o->precision == RAD_F32;
  a.cols = f32 ? (const void *)G.colsF : (const void *)G.cols;
  a.cols64 = G.cols;
  a.f1 = f32 ? (const void *)G.f1F : (const void *)G.f1;
  a.f2 = f32 ? (const void *)G.f2F : (const void *)G.f2;
  a.f3 = f32 ? (const void *)G.f3F : (const void *)G.f3;
  a.dir = ctx->dang.dir;
  a.dOmega = ctx->dang.dOmega;
  a.edge_geo = ctx->dang.edge_geo;
  a.perm = ctx->dang.perm;
  a.slot_nbr = ctx->dang.slot_nbr;
  a.slot_edge = ctx->dang.slot_edge;
  a.edge_pq = ctx->dang.edge_pq;
  a.edge_line = ctx->dang.edge_line;
  a.line_behind = ctx->dang.line_behind;
  a.n_edge = ctx->ang.n_edge;
  a.mapr_nb = ctx->dang.mapr_nb;
  a.mapr_minv = ctx->dang.mapr_minv;
  a.mapr_xo = ctx->dang.mapr_xo;
  a.mapr_xn = ctx->dang.mapr_xn;
  a.recon_ang = o->recon_ang;
  a.recon = o->recon;
  a.mode = o->coupling;
  a.zero_guard = o->zero_guard;
  a.n0crit = o->n0crit;
  a.a_rad = o->a_rad;
  a.gamma = o->gamma;
  a.inv_gm1 = 1.0 / (o->gamma - 1.0);
  a.tau_const = o->tau_const;
  a.err = ctx->err_word;
  for (int f = 0; f < 6; ++f) a.halo[f] = nullptr;
  a.divF = nullptr;
  return a;
}

int check_stage(const StageArgs &a, bool f32, std::string &err) {
  if (a.recon == RAD_RECON_PPM && a.ndim >= 2 && a.n2 < 3 &&
      (a.bc_lo[1] == RAD_BC_POLAR || a.bc_hi[1] == RAD_BC_POLAR)) {
    err = "PPM across a polar boundary needs at least three cells in x2";
    return RAD_EUNSUPPORTED;
  }
  if ((size_t)a.n1 * a.n2 * a.n3 * a.nap >= ((size_t)1 << 32)) {
    err = "more than 2^32 intensity elements in one block";
    return RAD_EUNSUPPORTED;
  }
  const int threads = (a.nap / 2 + 31) / 32 * 32;
  const bool mapr = a.recon_ang == RAD_RECON_MAPR;
  const size_t smem = f32 ? stage_smem<float, false>(threads, a.nap, a.kc, a.depth, a.tau_const > 0.0,
                                                     stage_rows(a.recon), mapr)
                          : stage_smem<double, false>(threads, a.nap, a.kc, a.depth, a.tau_const > 0.0,
                                                      stage_rows(a.recon), mapr);
  if (smem > (size_t)227 * 1024 || threads + 32 > kStageMaxThreads) {
    err = "the stencil pipeline of this many bins does not fit one CTA in this precision";
    return RAD_EUNSUPPORTED;
  }
  return RAD_OK;
}

int launch_stage_s(rad_ctx *ctx, int stage, void *I, const rad_gas *gas, double dt, const rad_opts *o,
                   double *gas_src, void *scratch_I, double *scratch_T, const void *const *halo, std::string &err) {
  StageArgs a = make_stage_args(ctx, gas, dt, o, gas_src);
  const bool f32 = o->precision == RAD_F32;
  const bool ang = ctx->geom.kind != RAD_MINK_CART;
  {
    const int rc = check_stage(a, f32, err);
    if (rc != RAD_OK) return rc;
  }
  if (halo)
    for (int f = 0; f < 6; ++f) a.halo[f] = halo[f];
  // rad_dom: each stage is the transport-only stage kernel (I* with the
  // guard applied, T- in Tout) followed by the coupling kernel with the
  // radiation-dominated velocity substitution, in place
  const bool rd = o->rad_dom != 0;
  if (rd) a.mode = RAD_COUPLE_NONE;
  cudaError_t ce;
  if (stage == 1) {
    // stage 1: I^0 -> I^1 (scratch), T^0 -> T^1 (scratch)
    a.Iprev = I;
    a.I0 = I;
    a.Iout = scratch_I;
    a.T0 = gas->T;
    a.T1 = nullptr;
    a.Tout = scratch_T;
    a.stage2 = 0;
    a.dts = dt;
    ce = launch_stage(a, f32, ang, ctx->stream);
    if (ce == cudaSuccess && rd) ce = launch_couple_rd(a, f32, scratch_T, scratch_T, ctx->stream);
  } else {
    // stage 2: I^1 (+ own I^0) -> I^2 written over I^0; T -> gas->T
    a.Iprev = scratch_I;
    a.I0 = I;
    a.Iout = I;
    a.T0 = gas->T;
    a.T1 = scratch_T;
    a.Tout = gas->T;
    a.stage2 = 1;
    a.dts = 0.5 * dt;
    ce = launch_stage(a, f32, ang, ctx->stream);
    if (ce == cudaSuccess && rd) ce = launch_couple_rd(a, f32, gas->T, gas->T, ctx->stream);
  }
  if (ce != cudaSuccess) {
    err = std::string(stage == 1 ? "stage 1" : "stage 2") + " launch failed: " + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

int launch_step_groups(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src,
                       void *scratch_I, double *scratch_T, void *D, std::string &err) {
  const bool f32 = o->precision == RAD_F32;
  const bool ang = ctx->geom.kind != RAD_MINK_CART;
  const DevGeom &G = ctx->geom;
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  const size_t gbytes = ncell * ctx->ang.n_ap * (f32 ? 4 : 8);      // one group's intensity array
  auto at = [&](const void *p, int g) { return (void *)((char *)p + g * gbytes); };
  for (int stage = 1; stage <= 2; ++stage) {
    const void *Iin = stage == 1 ? I : scratch_I;
    int st = launch_freq_div(ctx, Iin, D, o->precision, err);
    if (st != RAD_OK) return st;
    for (int g = 0; g < ctx->n_groups; ++g) {
      rad_gas gg = *gas;
      gg.alpha_a = gas->alpha_a ? gas->alpha_a + g * ncell : nullptr;
      gg.alpha_s = gas->alpha_s ? gas->alpha_s + g * ncell : nullptr;
      gg.eta = gas->eta ? gas->eta + g * ncell : nullptr;
      StageArgs a = make_stage_args(ctx, &gg, dt, o, gas_src ? gas_src + 4 * g * ncell : nullptr);
      if (g == 0 && stage == 1 && (st = check_stage(a, f32, err)) != RAD_OK) return st;
      a.divF = at(D, g);
      a.Iprev = at(Iin, g);
      a.I0 = at(I, g);
      a.Iout = stage == 1 ? at(scratch_I, g) : at(I, g);
      // the gas temperature is frozen (fixed-emissivity or no coupling): every
      // group writes the same values
      a.T0 = gas->T;
      a.T1 = stage == 1 ? nullptr : scratch_T;
      a.Tout = stage == 1 ? scratch_T : gas->T;
      a.stage2 = stage == 2;
      a.dts = stage == 1 ? dt : 0.5 * dt;
      const cudaError_t ce = launch_stage(a, f32, ang, ctx->stream);
      if (ce != cudaSuccess) {
        err = std::string("multigroup stage launch failed: ") + cudaGetErrorString(ce);
        return RAD_ECUDA;
      }
    }
  }
  return RAD_OK;
}

int launch_step(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src,
                void *scratch_I, double *scratch_T, std::string &err) {
  int st = launch_stage_s(ctx, 1, I, gas, dt, o, gas_src, scratch_I, scratch_T, nullptr, err);
  if (st == RAD_OK) st = launch_stage_s(ctx, 2, I, gas, dt, o, gas_src, scratch_I, scratch_T, nullptr, err);
  return st;
}

int launch_cfl(rad_ctx *ctx, double cfl, double *dt_out, std::string &err) {
  const DevGeom &G = ctx->geom;
  unsigned long long *d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
    err = "cfl: allocation failed";
    return RAD_ENOMEM;
  }
  unsigned long long init = (unsigned long long)0x7ff0000000000000ULL;   // +inf
  cudaMemcpyAsync(d, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream);
  double dx3 = G.xf[2][1] - G.xf[2][0];
  const double *xf1 = G.xf_dev, *xf2 = G.xf_dev + G.xf[0].size();
  int threads = (ctx->ang.n_ang + 31) / 32 * 32;
  k_cfl<<<G.n[0] * G.n[1], threads, 0, ctx->stream>>>(
      G.cols, G.n[0], G.n[1], G.ndim, xf1, xf2, dx3, ctx->ang.n_ang, ctx->dang.dir, ctx->dang.dOmega,
      ctx->dang.slot_nbr, ctx->dang.slot_edge, ctx->dang.edge_geo, G.kind != RAD_MINK_CART, ctx->nu_edges_dev,
      ctx->n_groups, d);
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  cudaError_t ce = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  if (ce != cudaSuccess) {
    err = std::string("cfl kernel failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  double best;
  std::memcpy(&best, &h, sizeof(best));
  *dt_out = cfl * best;
  return RAD_OK;
}

}  // namespace rad
