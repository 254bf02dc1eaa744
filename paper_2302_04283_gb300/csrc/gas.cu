// Gas update from the radiation source (end of Sec. 2.5: the coupling's
// change of R^0_mu is subtracted from the gas, which then recovers its
// primitive state).
//
// Ideal gas of rest-mass density rho, temperature T (k_B / (mu m_p) = 1:
// p = rho T) and tetrad-frame velocity u^ihat.  Conserved: D = rho u^0 and
// T^0_mu = w u^0 u_mu + p delta^0_mu with w = rho + Gamma p / (Gamma - 1).
// The source src_mu (rad_step's gas_src, -dR^0_mu) is added to T^0_mu at
// fixed D; in the normal observer's tetrad (e^0_ihat = 0) the new state has
//   D-hat = D / n^0,  E = -T^0_mu e^mu_0hat / n^0,  S_i = T^0_mu e^mu_ihat / n^0,
// and p solves f(p) = p - (Gamma-1)/Gamma (w(p) - D-hat (1 - v^2)^(1/2)) = 0
// with v = S / (E + p), w = (E + p)(1 - v^2).  f increases on [0, Gamma E]
// and changes sign there for every physical state (E > (S^2 + D-hat^2)^(1/2));
// it is solved by Newton's method from the old pressure, kept inside that
// bracket by bisection, in FP64.  One thread per cell.
#include <cmath>

#include "rad_internal.h"

namespace rad {

namespace {

__global__ void k_gas_update(const ColGeo *__restrict__ cols, int ncol, long long ncell, double *rho, double *u,
                             double *T, const double *__restrict__ src, int nsrc, double gam, int *err) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  const ColGeo &cg = cols[cell % ncol];
  const double r0 = rho[cell], T0 = T[cell];
  const double ua[4] = {sqrt(1.0 + u[3 * cell] * u[3 * cell] + u[3 * cell + 1] * u[3 * cell + 1] +
                             u[3 * cell + 2] * u[3 * cell + 2]),
                        u[3 * cell], u[3 * cell + 1], u[3 * cell + 2]};
  double umu[4], ulow[4];
  for (int m = 0; m < 4; ++m) {
    umu[m] = cg.e[m][0] * ua[0] + cg.e[m][1] * ua[1] + cg.e[m][2] * ua[2] + cg.e[m][3] * ua[3];
    ulow[m] = cg.M[m][0] * ua[0] + cg.M[m][1] * ua[1] + cg.M[m][2] * ua[2] + cg.M[m][3] * ua[3];
  }
  const double p0 = r0 * T0;
  const double gfac = (gam - 1.0) / gam;
  const double w0 = r0 + p0 / gfac;
  double Q[4];
  for (int m = 0; m < 4; ++m) Q[m] = w0 * umu[0] * ulow[m];
  Q[0] += p0;
  for (int s = 0; s < nsrc; ++s)
    for (int m = 0; m < 4; ++m) Q[m] += src[((size_t)s * ncell + cell) * 4 + m];
  const double n0 = cg.n0up;
  double Qt[4];
  for (int A = 0; A < 4; ++A) Qt[A] = (Q[0] * cg.e[0][A] + Q[1] * cg.e[1][A] + Q[2] * cg.e[2][A] + Q[3] * cg.e[3][A]) / n0;
  const double E = -Qt[0], S1 = Qt[1], S2 = Qt[2], S3 = Qt[3];
  const double Ss = S1 * S1 + S2 * S2 + S3 * S3;
  const double Dh = r0 * umu[0] / n0;
  if (!(E * E > Ss + Dh * Dh) || !(Dh > 0.0) || !(E > 0.0)) {
    atomicOr(err, kErrNoConv);
    return;
  }
  auto f = [&](double p, double &fp) {
    const double Ep = E + p;
    const double v2 = Ss / (Ep * Ep);
    const double sq = sqrt(1.0 - v2);
    fp = 1.0 - gfac * (1.0 + v2 - Dh * v2 / (Ep * sq));
    return p - gfac * ((Ep - Ss / Ep) - Dh * sq);
  };
  double lo = 0.0, hi = gam * E, p = fmin(fmax(p0, 0.0), hi), d;
  bool ok = false;
  for (int it = 0; it < 200; ++it) {
    const double fv = f(p, d);
    if (fv == 0.0) {
      ok = true;
      break;
    }
    if (fv < 0.0) lo = p;
    else hi = p;
    double pn = p - fv / d;
    if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
    if (fabs(pn - p) <= 1e-16 * fabs(pn) || hi - lo <= 1e-16 * hi) {
      p = pn;
      ok = true;
      break;
    }
    p = pn;
  }
  const double Ep = E + p;
  const double iv = 1.0 / Ep;
  const double v1 = S1 * iv, v2 = S2 * iv, v3 = S3 * iv;
  const double g = 1.0 / sqrt(1.0 - (v1 * v1 + v2 * v2 + v3 * v3));
  const double rn = Dh / g;
  if (!ok || !isfinite(p) || !(rn > 0.0)) {
    atomicOr(err, kErrNoConv);
    return;
  }
  rho[cell] = rn;
  T[cell] = p / rn;
  u[3 * cell] = g * v1;
  u[3 * cell + 1] = g * v2;
  u[3 * cell + 2] = g * v3;
}

}  // namespace

int launch_gas_update(rad_ctx *ctx, double *rho, double *u, double *T, const double *src, int nsrc, double gamma,
                      std::string &err) {
  const DevGeom &G = ctx->geom;
  const long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
  const int threads = 128;
  k_gas_update<<<(unsigned)((ncell + threads - 1) / threads), threads, 0, ctx->stream>>>(
      G.cols, G.n[0] * G.n[1], ncell, rho, u, T, src, nsrc, gamma, ctx->err_word);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("gas update launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
