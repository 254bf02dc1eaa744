// C ABI entry points: argument validation, context state, table upload and
// dispatch to the kernels.  No exception crosses this boundary.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "rad_internal.h"

using rad::AngleGrid;

namespace {

int fail(rad_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

void free_angles(rad::DevAngles &d) {
  cudaFree(d.dir);
  cudaFree(d.dOmega);
  cudaFree(d.slot_nbr);
  cudaFree(d.slot_edge);
  cudaFree(d.perm);
  cudaFree(d.edge_geo);
  cudaFree(d.edge_pq);
  cudaFree(d.edge_line);
  cudaFree(d.line_behind);
  cudaFree(d.mapr_nb);
  cudaFree(d.mapr_minv);
  cudaFree(d.mapr_xo);
  cudaFree(d.mapr_xn);
  d = rad::DevAngles();
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src, cudaStream_t st) {
  cudaError_t e = cudaMalloc(dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

int rad_create(rad_ctx **out, void *cuda_stream) {
  if (!out) return RAD_EINVAL;
  *out = nullptr;
  rad_ctx *c = new (std::nothrow) rad_ctx();
  if (!c) return RAD_ENOMEM;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaMalloc(&c->err_word, sizeof(int)) != cudaSuccess) {
    delete c;
    return RAD_ENOMEM;
  }
  cudaMemsetAsync(c->err_word, 0, sizeof(int), c->stream);
  *out = c;
  return RAD_OK;
}

void rad_destroy(rad_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_angles(ctx->dang);
  rad::free_geometry(ctx->geom);
  cudaFree(ctx->err_word);
  cudaFree(ctx->scratch_I);
  cudaFree(ctx->scratch_T);
  cudaFree(ctx->adj_buf);
  cudaFree(ctx->wt_dev);
  cudaFree(ctx->loss_buf);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamSynchronize(ctx->back_stream);
    cudaStreamSynchronize(ctx->mom_stream);
    cudaStreamDestroy(ctx->copy_stream);
    cudaStreamDestroy(ctx->back_stream);
    cudaStreamDestroy(ctx->mom_stream);
    for (int s = 0; s < rad_ctx::kHostSlots; ++s) {
      cudaEventDestroy(ctx->ev_h2d[s]);
      cudaEventDestroy(ctx->ev_step[s]);
      cudaEventDestroy(ctx->ev_done[s]);
      cudaEventDestroy(ctx->ev_back[s]);
    }
  }
  cudaFree(ctx->host_slot_buf);
  cudaFree(ctx->nu_edges_dev);
  cudaFree(ctx->freq_buf);
  delete ctx;
}

const char *rad_last_error(const rad_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

void rad_opts_default(rad_opts *o) {
  if (!o) return;
  o->precision = RAD_F64;
  o->recon = RAD_RECON_PLM;
  o->coupling = RAD_COUPLE_THERMAL;
  o->n0crit = 0.1;
  o->zero_guard = 1;
  o->a_rad = 1.0;
  o->gamma = 5.0 / 3.0;
  o->tau_const = 0.0;
  o->rad_dom = 0;
  o->recon_ang = RAD_RECON_DC;
}

// Upload a built angle grid and make it the context's (the metric must be
// set again afterwards).
static int install_angles(rad_ctx *ctx, AngleGrid &g, int *n_ang_out, int *n_ang_padded_out) {
  cudaStreamSynchronize(ctx->stream);
  free_angles(ctx->dang);
  cudaFree(ctx->wt_dev);
  ctx->wt_dev = nullptr;
  ctx->have_angles = ctx->have_metric = false;
  // device tables, padded to n_ap bins with zero directions / solid angles
  std::vector<double> dir(3 * g.n_ap, 0.0), dOm(g.n_ap, 0.0), egeo(8 * g.n_edge, 0.0);
  std::vector<int> snb(6 * g.n_ap, -1), sed(6 * g.n_ap, -1), perm(g.n_ap, 0);
  std::vector<int> lbh(g.line_behind.empty() ? 0 : rad::kMaxBehind * g.n_ap, -1);   // padded bins: none
  for (size_t q = 0; q < g.line_behind.size(); ++q) lbh[q] = g.line_behind[q];
  // minimum-angle plane tables, padded to n_ap bins (padding: no neighbours)
  const bool mapr = !g.mapr_nb.empty();
  std::vector<int> mnb(mapr ? 6 * g.n_ap : 0, -1);
  std::vector<double> mminv(mapr ? 24 * g.n_ap : 0, 0.0), mxo(mapr ? 12 * g.n_ap : 0, 0.0),
      mxn(mapr ? 12 * g.n_ap : 0, 0.0);
  for (size_t q = 0; q < g.mapr_nb.size(); ++q) mnb[q] = g.mapr_nb[q];
  for (size_t q = 0; q < g.mapr_minv.size(); ++q) mminv[q] = g.mapr_minv[q];
  for (size_t q = 0; q < g.mapr_xo.size(); ++q) mxo[q] = g.mapr_xo[q];
  for (size_t q = 0; q < g.mapr_xn.size(); ++q) mxn[q] = g.mapr_xn[q];
  for (int n = 0; n < g.n_ang; ++n) {
    for (int a = 0; a < 3; ++a) dir[3 * n + a] = g.dir[3 * n + a];
    dOm[n] = g.dOmega[n];
    for (int s = 0; s < 6; ++s) {
      snb[6 * n + s] = g.nbr[6 * n + s];
      sed[6 * n + s] = g.slot_edge[6 * n + s];
    }
    perm[n] = g.perm[n];
  }
  for (int e = 0; e < g.n_edge; ++e) {
    for (int a = 0; a < 3; ++a) {
      egeo[8 * e + a] = g.edge_mid[3 * e + a];
      egeo[8 * e + 3 + a] = g.edge_nrm[3 * e + a];
    }
    egeo[8 * e + 6] = g.edge_len[e];
    egeo[8 * e + 7] = g.edge_pq[2 * e];
  }
  cudaError_t ce;
  if ((ce = upload(&ctx->dang.dir, dir, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.dOmega, dOm, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.slot_nbr, snb, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.slot_edge, sed, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.perm, perm, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.edge_geo, egeo, ctx->stream)) != cudaSuccess ||
      (ce = upload(&ctx->dang.edge_pq, g.edge_pq, ctx->stream)) != cudaSuccess ||
      (!g.edge_line.empty() && (ce = upload(&ctx->dang.edge_line, g.edge_line, ctx->stream)) != cudaSuccess) ||
      (!lbh.empty() && (ce = upload(&ctx->dang.line_behind, lbh, ctx->stream)) != cudaSuccess) ||
      (mapr && ((ce = upload(&ctx->dang.mapr_nb, mnb, ctx->stream)) != cudaSuccess ||
                (ce = upload(&ctx->dang.mapr_minv, mminv, ctx->stream)) != cudaSuccess ||
                (ce = upload(&ctx->dang.mapr_xo, mxo, ctx->stream)) != cudaSuccess ||
                (ce = upload(&ctx->dang.mapr_xn, mxn, ctx->stream)) != cudaSuccess))) {
    free_angles(ctx->dang);
    return fail(ctx, RAD_ENOMEM, std::string("angle table upload failed: ") + cudaGetErrorString(ce));
  }
  if ((ce = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return fail(ctx, RAD_ECUDA, std::string("angle table upload failed: ") + cudaGetErrorString(ce));
  ctx->ang = std::move(g);
  ctx->have_angles = true;
  if (n_ang_out) *n_ang_out = ctx->ang.n_ang;
  if (n_ang_padded_out) *n_ang_padded_out = ctx->ang.n_ap;
  return RAD_OK;
}

int rad_init_angles(rad_ctx *ctx, int level, int *n_ang_out, int *n_ang_padded_out) {
  if (!ctx) return RAD_EINVAL;
  AngleGrid g;
  std::string err;
  if (!rad::build_geodesic(level, g, err)) return fail(ctx, RAD_EINVAL, err);
  return install_angles(ctx, g, n_ang_out, n_ang_padded_out);
}

int rad_init_angles_latlong(rad_ctx *ctx, int n_zeta, int n_psi, int *n_ang_out, int *n_ang_padded_out) {
  if (!ctx) return RAD_EINVAL;
  AngleGrid g;
  std::string err;
  if (!rad::build_latlong(n_zeta, n_psi, g, err)) return fail(ctx, RAD_EINVAL, err);
  return install_angles(ctx, g, n_ang_out, n_ang_padded_out);
}

int rad_get_angles(rad_ctx *ctx, double *dir, double *dOmega, int *nbr) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_angles) return fail(ctx, RAD_ESTATE, "rad_init_angles has not been called");
  const AngleGrid &g = ctx->ang;
  if (dir) std::memcpy(dir, g.dir.data(), g.dir.size() * sizeof(double));
  if (dOmega) std::memcpy(dOmega, g.dOmega.data(), g.dOmega.size() * sizeof(double));
  if (nbr) std::memcpy(nbr, g.nbr.data(), g.nbr.size() * sizeof(int));
  return RAD_OK;
}

int rad_set_metric(rad_ctx *ctx, const rad_metric *m, const rad_grid *gr) {
  if (!ctx) return RAD_EINVAL;
  if (!m || !gr) return fail(ctx, RAD_EINVAL, "null metric or grid");
  if (!ctx->have_angles) return fail(ctx, RAD_ESTATE, "rad_init_angles must precede rad_set_metric");
  if (m->kind < RAD_MINK_CART || m->kind > RAD_KS_SPH) return fail(ctx, RAD_EINVAL, "unknown metric kind");
  if (m->kind == RAD_KS_SPH && !(std::fabs(m->spin) < 1.0)) return fail(ctx, RAD_EINVAL, "|spin| must be < 1");
  if (gr->ndim < 1 || gr->ndim > 3) return fail(ctx, RAD_EINVAL, "ndim must be 1, 2 or 3");
  for (int d = 0; d < 3; ++d) {
    if (gr->n[d] < 1) return fail(ctx, RAD_EINVAL, "cell counts must be >= 1");
    if (d >= gr->ndim && gr->n[d] != 1) return fail(ctx, RAD_EINVAL, "n[d] must be 1 beyond ndim");
    if (!gr->xf[d]) return fail(ctx, RAD_EINVAL, "null face coordinates");
    for (int t = 0; t < gr->n[d]; ++t)
      if (!(gr->xf[d][t + 1] > gr->xf[d][t])) return fail(ctx, RAD_EINVAL, "face coordinates must increase");
    for (int s = 0; s < 2; ++s) {
      int bc = s ? gr->bc_hi[d] : gr->bc_lo[d];
      if (bc < RAD_BC_PERIODIC || bc > RAD_BC_HALO) return fail(ctx, RAD_EINVAL, "unknown boundary kind");
      if (bc == RAD_BC_HALO && d >= gr->ndim) return fail(ctx, RAD_EINVAL, "a shared face needs a flux dimension");
      if (bc == RAD_BC_HALO && gr->n[d] < rad::kHaloLayers)
        return fail(ctx, RAD_EINVAL, "a block needs at least 3 cells across a shared face");
      if (bc == RAD_BC_POLAR && (d != 1 || m->kind == RAD_MINK_CART))
        return fail(ctx, RAD_EINVAL, "polar boundaries apply to theta (x2) of a spherical metric only");
    }
    if ((gr->bc_lo[d] == RAD_BC_PERIODIC) != (gr->bc_hi[d] == RAD_BC_PERIODIC))
      return fail(ctx, RAD_EINVAL, "periodic boundaries must be set on both sides");
  }
  const double *x3 = gr->xf[2];
  double w3 = x3[1] - x3[0];
  for (int t = 1; t < gr->n[2]; ++t)
    if (std::fabs((x3[t + 1] - x3[t]) - w3) > 1e-12 * std::fabs(w3))
      return fail(ctx, RAD_EUNSUPPORTED, "x3 faces must be uniformly spaced");
  bool polar = gr->bc_lo[1] == RAD_BC_POLAR || gr->bc_hi[1] == RAD_BC_POLAR;
  if (polar && (gr->bc_lo[2] == RAD_BC_HALO || gr->bc_hi[2] == RAD_BC_HALO))
    return fail(ctx, RAD_EUNSUPPORTED, "a block on a polar axis must hold the whole phi range (no shared x3 faces)");
  if (polar) {
    if (gr->n[1] < 2) return fail(ctx, RAD_EINVAL, "polar boundaries need n[1] >= 2");
    if (gr->n[2] > 1 && (gr->n[2] % 2 != 0)) return fail(ctx, RAD_EINVAL, "polar boundaries need an even n[2]");
    if (std::fabs((x3[gr->n[2]] - x3[0]) - 2.0 * rad::kPi) > 1e-9)
      return fail(ctx, RAD_EINVAL, "polar boundaries need x3 to span 2 pi");
    if (gr->bc_lo[1] == RAD_BC_POLAR && std::fabs(gr->xf[1][0]) > 1e-12)
      return fail(ctx, RAD_EINVAL, "polar boundary at x2 lo needs theta = 0");
    if (gr->bc_hi[1] == RAD_BC_POLAR && std::fabs(gr->xf[1][gr->n[1]] - rad::kPi) > 1e-12)
      return fail(ctx, RAD_EINVAL, "polar boundary at x2 hi needs theta = pi");
  }
  if (m->kind != RAD_MINK_CART) {
    if (!(gr->xf[0][0] > 0.0)) return fail(ctx, RAD_EINVAL, "r must be positive");
    if (gr->xf[1][0] < 0.0 || gr->xf[1][gr->n[1]] > rad::kPi + 1e-12) return fail(ctx, RAD_EINVAL, "theta outside [0, pi]");
    if (m->kind == RAD_KS_SPH) {
      double rh = 1.0 + std::sqrt(1.0 - m->spin * m->spin);
      (void)rh;   // Kerr-Schild coordinates are regular through the horizon
    }
  }
  rad::DevGeom &G = ctx->geom;
  G.kind = m->kind;
  G.spin = m->kind == RAD_KS_SPH ? m->spin : 0.0;
  G.ndim = gr->ndim;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = gr->n[d];
    G.bc_lo[d] = gr->bc_lo[d];
    G.bc_hi[d] = gr->bc_hi[d];
    G.xf[d].assign(gr->xf[d], gr->xf[d] + gr->n[d] + 1);
  }
  std::string err;
  ctx->have_metric = false;
  int st = rad::compute_geometry(ctx, err);
  if (st != RAD_OK) return fail(ctx, st, err);
  ctx->have_metric = true;
  return RAD_OK;
}

int rad_cfl_dt(rad_ctx *ctx, double cfl, double *dt_out) {
  if (!ctx) return RAD_EINVAL;
  if (!dt_out || !(cfl > 0.0)) return fail(ctx, RAD_EINVAL, "cfl must be > 0 and dt_out non-null");
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  std::string err;
  int st = rad::launch_cfl(ctx, cfl, dt_out, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

static int check_gas(rad_ctx *ctx, const rad_gas *gas, const rad_opts *o, bool need_T) {
  if (!gas) return fail(ctx, RAD_EINVAL, "null gas");
  if (o->coupling != RAD_COUPLE_NONE) {
    if (!gas->rho || !gas->u || !gas->alpha_a || !gas->alpha_s)
      return fail(ctx, RAD_EINVAL, "gas fields rho, u, alpha_a, alpha_s are required for coupling");
    if (o->coupling == RAD_COUPLE_EMISSIVITY && !gas->eta)
      return fail(ctx, RAD_EINVAL, "emissivity coupling needs gas->eta");
  }
  if (o->tau_const > 0.0 && (!gas->u || !gas->alpha_a || !gas->alpha_s))
    return fail(ctx, RAD_EINVAL, "the optical-depth flux weighting needs gas u, alpha_a, alpha_s");
  if (need_T && !gas->T) return fail(ctx, RAD_EINVAL, "gas->T is required");
  return RAD_OK;
}

static int check_opts(rad_ctx *ctx, const rad_opts *o) {
  if (!o) return fail(ctx, RAD_EINVAL, "null opts");
  if (o->precision != RAD_F64 && o->precision != RAD_F32) return fail(ctx, RAD_EINVAL, "bad precision");
  if (o->recon != RAD_RECON_DC && o->recon != RAD_RECON_PLM && o->recon != RAD_RECON_PPM)
    return fail(ctx, RAD_EINVAL, "bad recon");
  if (o->coupling < RAD_COUPLE_THERMAL || o->coupling > RAD_COUPLE_NONE) return fail(ctx, RAD_EINVAL, "bad coupling");
  if (o->coupling == RAD_COUPLE_THERMAL && !(o->gamma > 1.0)) return fail(ctx, RAD_EINVAL, "gamma must be > 1");
  if (!(o->n0crit >= 0.0)) return fail(ctx, RAD_EINVAL, "n0crit must be >= 0");
  if (!(o->tau_const >= 0.0) || !std::isfinite(o->tau_const))
    return fail(ctx, RAD_EINVAL, "tau_const must be finite and >= 0");
  if (o->rad_dom != 0 && o->rad_dom != 1) return fail(ctx, RAD_EINVAL, "rad_dom must be 0 or 1");
  if (o->recon_ang != RAD_RECON_DC && o->recon_ang != RAD_RECON_PLM && o->recon_ang != RAD_RECON_MAPR)
    return fail(ctx, RAD_EINVAL, "bad recon_ang");
  if (o->recon_ang == RAD_RECON_PLM && ctx->ang.edge_line.empty())
    return fail(ctx, RAD_EUNSUPPORTED, "angular PLM needs a latitude-longitude grid (rad_init_angles_latlong)");
  if (o->recon_ang == RAD_RECON_MAPR && ctx->ang.mapr_nb.empty())
    return fail(ctx, RAD_EUNSUPPORTED, "MAPR needs a geodesic grid (rad_init_angles)");
  if (o->rad_dom && o->coupling != RAD_COUPLE_THERMAL)
    return fail(ctx, RAD_EINVAL, "rad_dom applies to the thermal coupling");
  return RAD_OK;
}

}  // extern "C"

// The host-side checks every RK2 step entry (rad_step, rad_step_noalloc)
// makes before anything is launched: options, gas fields, the intensity
// pointer, dt, the bin count and the 32-bit element index.
static bool has_halo(const rad::DevGeom &G) {
  for (int d = 0; d < 3; ++d)
    if (G.bc_lo[d] == RAD_BC_HALO || G.bc_hi[d] == RAD_BC_HALO) return true;
  return false;
}

int rad::check_step_args(rad_ctx *ctx, const void *I, const rad_gas *gas, double dt, const rad_opts *o,
                         bool staged) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (!staged && has_halo(ctx->geom))
    return fail(ctx, RAD_ESTATE, "a block with faces shared with other blocks (RAD_BC_HALO) steps with rad_step_stage");
  int st = check_opts(ctx, o);
  if (st != RAD_OK) return st;
  if (has_halo(ctx->geom) && o->tau_const > 0.0)
    return fail(ctx, RAD_EUNSUPPORTED, "the optical-depth weighting reads the neighbour's gas: single blocks only");
  if (ctx->n_groups > 0) {
    if (staged) return fail(ctx, RAD_EUNSUPPORTED, "multigroup transport steps single blocks with rad_step");
    if (o->coupling == RAD_COUPLE_THERMAL || o->rad_dom)
      return fail(ctx, RAD_EUNSUPPORTED, "multigroup transport couples with fixed emissivity or not at all");
  }
  if ((st = check_gas(ctx, gas, o, true)) != RAD_OK) return st;
  if (!I || !aligned16(I)) return fail(ctx, RAD_EINVAL, "I must be a 16-byte aligned device pointer");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, RAD_EINVAL, "dt must be finite and > 0");
  if (ctx->ang.n_ang > rad::kMaxBinsStep)
    return fail(ctx, RAD_EUNSUPPORTED, "the step supports up to 812 bins (geodesic level 9)");
  const rad::DevGeom &G = ctx->geom;
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  if (ncell * ctx->ang.n_ap >= ((size_t)1 << 32))
    return fail(ctx, RAD_EUNSUPPORTED, "the step handles fewer than 2^32 intensity elements in one block");
  return RAD_OK;
}

extern "C" {

// The stage scratch of rad_step / rad_step_stage (one intensity array and one
// temperature per cell), grown on demand.
static int ensure_scratch(rad_ctx *ctx, const rad_opts *o) {
  const rad::DevGeom &G = ctx->geom;
  size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  size_t esz = o->precision == RAD_F32 ? 4 : 8;
  size_t need = ncell * ctx->ang.n_ap * esz * (size_t)std::max(1, ctx->n_groups);
  if (ctx->n_groups > 0 && ctx->freq_bytes < need) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->freq_buf);
    ctx->freq_buf = nullptr;
    ctx->freq_bytes = 0;
    if (cudaMalloc(&ctx->freq_buf, need) != cudaSuccess) return fail(ctx, RAD_ENOMEM, "frequency scratch allocation failed");
    ctx->freq_bytes = need;
  }
  if (ctx->scratch_I_bytes < need) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->scratch_I);
    ctx->scratch_I = nullptr;
    ctx->scratch_I_bytes = 0;
    if (cudaMalloc(&ctx->scratch_I, need) != cudaSuccess) return fail(ctx, RAD_ENOMEM, "stage scratch allocation failed");
    ctx->scratch_I_bytes = need;
  }
  if (ctx->scratch_T_count < ncell) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->scratch_T);
    ctx->scratch_T = nullptr;
    ctx->scratch_T_count = 0;
    if (cudaMalloc(&ctx->scratch_T, ncell * sizeof(double)) != cudaSuccess)
      return fail(ctx, RAD_ENOMEM, "stage scratch allocation failed");
    ctx->scratch_T_count = ncell;
  }
  return RAD_OK;
}

int rad_step(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *o, double *gas_src) {
  int st = rad::check_step_args(ctx, I, gas, dt, o);
  if (st != RAD_OK) return st;
  if ((st = ensure_scratch(ctx, o)) != RAD_OK) return st;
  ctx->stage1_prec = -1;    // the scratch no longer holds a rad_step_stage stage-1 result
  std::string err;
  if (ctx->n_groups > 0)
    st = rad::launch_step_groups(ctx, I, gas, dt, o, gas_src, ctx->scratch_I, ctx->scratch_T, ctx->freq_buf, err);
  else
    st = rad::launch_step(ctx, I, gas, dt, o, gas_src, ctx->scratch_I, ctx->scratch_T, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_step_stage(rad_ctx *ctx, int stage, void *I, const rad_gas *gas, double dt, const rad_opts *o,
                   double *gas_src, const void *const *halo) {
  int st = rad::check_step_args(ctx, I, gas, dt, o, true);
  if (st != RAD_OK) return st;
  if (stage != 1 && stage != 2) return fail(ctx, RAD_EINVAL, "stage must be 1 or 2");
  const rad::DevGeom &G = ctx->geom;
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side)
      if ((side ? G.bc_hi[d] : G.bc_lo[d]) == RAD_BC_HALO && (!halo || !halo[2 * d + side] ||
                                                               !aligned16(halo[2 * d + side])))
        return fail(ctx, RAD_EINVAL, "every shared face needs a 16-byte aligned halo buffer");
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  const size_t esz = o->precision == RAD_F32 ? 4 : 8;
  if (stage == 1) {
    if ((st = ensure_scratch(ctx, o)) != RAD_OK) return st;
    ctx->stage1_prec = o->precision;
  } else if (ctx->stage1_prec != o->precision || ctx->scratch_I_bytes < ncell * ctx->ang.n_ap * esz ||
             ctx->scratch_T_count < ncell) {
    return fail(ctx, RAD_ESTATE, "stage 2 needs a stage 1 of the same precision on this context first");
  }
  std::string err;
  st = rad::launch_stage_s(ctx, stage, I, gas, dt, o, gas_src, ctx->scratch_I, ctx->scratch_T, halo, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_gas_update(rad_ctx *ctx, double *rho, double *u, double *T, const double *src, int n_src, double gamma) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (!rho || !u || !T || !src) return fail(ctx, RAD_EINVAL, "null argument");
  if (n_src < 1) return fail(ctx, RAD_EINVAL, "n_src must be >= 1");
  if (!(gamma > 1.0) || !(gamma <= 2.0)) return fail(ctx, RAD_EINVAL, "gamma must be in (1, 2]");
  std::string err;
  int st = rad::launch_gas_update(ctx, rho, u, T, src, n_src, gamma, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_set_groups(rad_ctx *ctx, int n_groups, const double *nu_edges) {
  if (!ctx) return RAD_EINVAL;
  if (n_groups < 0 || n_groups > 4096 || (n_groups > 0 && !nu_edges))
    return fail(ctx, RAD_EINVAL, "n_groups must be in 0..4096 with n_groups + 1 edges");
  for (int g = 0; g < n_groups; ++g)
    if (!(nu_edges[g + 1] > nu_edges[g]) || !std::isfinite(nu_edges[g]))
      return fail(ctx, RAD_EINVAL, "edges must increase and be finite except the last");
  if (n_groups > 0 && !(nu_edges[0] >= 0.0)) return fail(ctx, RAD_EINVAL, "the lowest edge must be >= 0");
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->nu_edges_dev);
  ctx->nu_edges_dev = nullptr;
  ctx->nu_edges.clear();
  ctx->n_groups = 0;
  if (n_groups == 0) return RAD_OK;
  ctx->nu_edges.assign(nu_edges, nu_edges + n_groups + 1);
  cudaError_t ce = upload(&ctx->nu_edges_dev, ctx->nu_edges, ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return fail(ctx, RAD_ENOMEM, std::string("group edge upload failed: ") + cudaGetErrorString(ce));
  ctx->n_groups = n_groups;
  return RAD_OK;
}

int rad_halo_pack(rad_ctx *ctx, const void *I, int precision, int dim, int side, void *buf) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (precision != RAD_F64 && precision != RAD_F32) return fail(ctx, RAD_EINVAL, "bad precision");
  if (dim < 0 || dim >= ctx->geom.ndim || (side != 0 && side != 1))
    return fail(ctx, RAD_EINVAL, "dim must be a flux dimension and side 0 or 1");
  if (ctx->geom.n[dim] < rad::kHaloLayers) return fail(ctx, RAD_EINVAL, "fewer than 3 cells across the face");
  if (!buf || !aligned16(buf) || (I && !aligned16(I))) return fail(ctx, RAD_EINVAL, "buffers must be 16-byte aligned");
  if (!I) {
    const rad::DevGeom &G = ctx->geom;
    const size_t need = (size_t)G.n[0] * G.n[1] * G.n[2] * ctx->ang.n_ap * (precision == RAD_F32 ? 4 : 8);
    if (!ctx->scratch_I || ctx->scratch_I_bytes < need || ctx->stage1_prec != precision)
      return fail(ctx, RAD_ESTATE, "no stage-1 result of this precision on this context");
    I = ctx->scratch_I;
  }
  std::string err;
  int st = rad::launch_halo_pack(ctx, I, precision, dim, side, buf, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_moments(rad_ctx *ctx, const void *I, int precision, int frame, int method, const rad_gas *gas, void *R) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (!I || !R) return fail(ctx, RAD_EINVAL, "null I or R");
  if (precision != RAD_F64 && precision != RAD_F32) return fail(ctx, RAD_EINVAL, "bad precision");
  if (frame < RAD_FRAME_TETRAD || frame > RAD_FRAME_FLUID) return fail(ctx, RAD_EINVAL, "bad frame");
  if (method != RAD_MOM_SIMT && method != RAD_MOM_BF16X3) return fail(ctx, RAD_EINVAL, "bad method");
  if (method == RAD_MOM_BF16X3 && precision != RAD_F32)
    return fail(ctx, RAD_EINVAL, "the split-bf16 moments read float intensities");
  if (frame == RAD_FRAME_FLUID && (!gas || !gas->u)) return fail(ctx, RAD_EINVAL, "fluid frame needs gas->u");
  if (!aligned16(I) || !aligned16(R)) return fail(ctx, RAD_EINVAL, "I and R must be 16-byte aligned");
  std::string err;
  int st = rad::launch_moments(ctx, I, precision, frame, method, gas, R, ctx->stream, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_step_adjoint(rad_ctx *ctx, const void *I_n, const rad_gas *gas, double dt, const rad_opts *o,
                     const void *lam_np1, void *lam_n, const double *lamT_np1, double *lamT_n, double *g_aa,
                     double *g_as, double *g_eta) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  int st = check_opts(ctx, o);
  if (st != RAD_OK) return st;
  if ((st = check_gas(ctx, gas, o, true)) != RAD_OK) return st;
  if (has_halo(ctx->geom)) return fail(ctx, RAD_EUNSUPPORTED, "the adjoint steps single blocks (no RAD_BC_HALO faces)");
  if (ctx->n_groups > 0) return fail(ctx, RAD_EUNSUPPORTED, "the adjoint covers gray transport (no groups)");
  if (!I_n || !lam_np1 || !lam_n || !g_aa || !g_as) return fail(ctx, RAD_EINVAL, "null argument");
  if (!(dt > 0.0)) return fail(ctx, RAD_EINVAL, "dt must be > 0");
  if (ctx->ang.n_ang > rad::kMaxBinsStep)
    return fail(ctx, RAD_EUNSUPPORTED, "rad_step_adjoint supports up to 812 bins (geodesic level 9)");
  std::string err;
  st = rad::launch_adjoint(ctx, I_n, gas, dt, o, lam_np1, lam_n, lamT_np1, lamT_n, g_aa, g_as, g_eta, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_loss_outer(rad_ctx *ctx, const void *I, int precision, double *L_dev, void *dL_dI) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (!I || !L_dev) return fail(ctx, RAD_EINVAL, "null argument");
  if (precision != RAD_F64 && precision != RAD_F32) return fail(ctx, RAD_EINVAL, "bad precision");
  std::string err;
  int st = rad::launch_loss(ctx, I, precision, L_dev, dL_dI, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}

int rad_selftest_wait(rad_ctx *ctx, double seconds) {
  if (!ctx) return RAD_EINVAL;
  if (!(seconds > 0.0 && seconds <= 10.0)) return fail(ctx, RAD_EINVAL, "seconds must be in (0, 10]");
  const cudaError_t ce = rad::launch_wait_selftest(ctx, seconds);
  if (ce != cudaSuccess) return fail(ctx, RAD_ECUDA, std::string("self-test launch failed: ") + cudaGetErrorString(ce));
  return RAD_OK;
}

int rad_check(rad_ctx *ctx) {
  if (!ctx) return RAD_EINVAL;
  int h = 0;
  cudaError_t ce = cudaMemcpyAsync(&h, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(ctx->err_word, 0, sizeof(int), ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return fail(ctx, RAD_ECUDA, std::string("rad_check: ") + cudaGetErrorString(ce));
  if (h & (1 << 3)) return fail(ctx, RAD_ECUDA, "a device wait timed out (stage pipeline or tensor-core moments)");
  if (h & rad::kErrNoConv) return fail(ctx, RAD_ENOCONV, "a cell's quartic had no bracketed root or did not converge");
  if (h & rad::kErrNonFinite) return fail(ctx, RAD_ENONFINITE, "a non-finite intensity was produced");
  if (h & rad::kErrState)
    return fail(ctx, RAD_ESTATE, "the stage kernel met a bin pair with opposite upwind sides (angle numbering)");
  return RAD_OK;
}

}  // extern "C"
