// Frequency fluxes of multigroup transport (Sec. 2.2, Eq.
// radiation_integral_frequency): per cell, bin and group edge nu_f,
//   F_f = n^nu n_0 I_nu = nu_f s n_0 I_up / dnu_up,   s = n^nu / nu = -omega^0hat_{AB} n^A n^B,
// donor cell in frequency (the lower group where s > 0, the upper one where
// s < 0); the end edges let radiation out of the resolved range and none in,
// and an edge at nu = 0 or nu = infinity carries nothing.  The kernel writes
// each group's divergence F_{g+1} - F_g, which the stage kernel adds to the
// spatial and angular divergences of that group before the stage update.
//
// One CTA per cell; each thread owns one bin and walks the groups, carrying
// the flux of the previous edge, so every intensity is read once and every
// divergence written once (coalesced rows of n_ap elements).
#include <cmath>

#include "rad_internal.h"

namespace rad {

namespace {

template <typename R, typename Col>
__global__ void k_freq_div(const R *__restrict__ I, R *__restrict__ D, const Col *__restrict__ cols,
                           const double *__restrict__ dir, const double *__restrict__ edges, int ngroup,
                           int nang, int nap, int ncol, long long ncell) {
  const long long cell = blockIdx.x;
  for (int n = threadIdx.x; n < nap; n += blockDim.x) {
    const size_t gstride = (size_t)ncell * nap;
    const size_t off = (size_t)cell * nap + n;
    if (n >= nang) {
      for (int g = 0; g < ngroup; ++g) D[g * gstride + off] = R(0);
      continue;
    }
    const Col &cg = cols[cell % ncol];
    const R x = (R)dir[3 * n], y = (R)dir[3 * n + 1], z = (R)dir[3 * n + 2];
    const R pr[10] = {R(1), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
    R q0 = R(0);
#pragma unroll
    for (int p = 0; p < 10; ++p) q0 += (R)cg.K0[p] * pr[p];
    const R s = -q0;                                                     // n^nu / nu
    const R n0 = (R)cg.M[0][0] + (R)cg.M[0][1] * x + (R)cg.M[0][2] * y + (R)cg.M[0][3] * z;
    const R sn0 = s * n0;
    // mean specific intensity of group g (0 for a group reaching infinity)
    auto mean = [&](int g) -> R {
      const double dnu = edges[g + 1] - edges[g];
      return isinf(dnu) ? R(0) : I[g * gstride + off] / (R)dnu;
    };
    auto flux = [&](int f, R below, R above) -> R {
      const double nu = edges[f];
      if (nu == 0.0 || isinf(nu)) return R(0);
      return (R)nu * sn0 * (s > R(0) ? below : above);
    };
    R m_lo = R(0);
    R m_hi = mean(0);
    R F = flux(0, R(0), m_hi);
    for (int g = 0; g < ngroup; ++g) {
      m_lo = m_hi;
      m_hi = g + 1 < ngroup ? mean(g + 1) : R(0);
      const R Fn = flux(g + 1, m_lo, m_hi);
      D[g * gstride + off] = Fn - F;
      F = Fn;
    }
  }
}

}  // namespace

int launch_freq_div(rad_ctx *ctx, const void *I, void *D, int precision, std::string &err) {
  const DevGeom &G = ctx->geom;
  const long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
  const int ncol = G.n[0] * G.n[1];
  const int threads = std::min(256, (ctx->ang.n_ap + 31) / 32 * 32);
  if (precision == RAD_F32)
    k_freq_div<float, ColGeoF><<<(unsigned)ncell, threads, 0, ctx->stream>>>(
        (const float *)I, (float *)D, G.colsF, ctx->dang.dir, ctx->nu_edges_dev, ctx->n_groups, ctx->ang.n_ang,
        ctx->ang.n_ap, ncol, ncell);
  else
    k_freq_div<double, ColGeo><<<(unsigned)ncell, threads, 0, ctx->stream>>>(
        (const double *)I, (double *)D, G.cols, ctx->dang.dir, ctx->nu_edges_dev, ctx->n_groups, ctx->ang.n_ang,
        ctx->ang.n_ap, ncol, ncell);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("frequency flux launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
