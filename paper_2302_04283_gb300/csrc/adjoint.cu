// Reverse-mode step and the outgoing-flux loss.
#include "rad_internal.h"

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
    atomicAdd(L, s);
  }
}

int launch_loss(rad_ctx *ctx, const void *I, int precision, double *L, void *dL, std::string &err) {
  const DevGeom &G = ctx->geom;
  size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  size_t esz = precision == RAD_F32 ? 4 : 8;
  cudaMemsetAsync(L, 0, sizeof(double), ctx->stream);
  if (dL) cudaMemsetAsync(dL, 0, ncell * ctx->ang.n_ap * esz, ctx->stream);
  unsigned rows = (unsigned)(G.n[1] * G.n[2]);
  if (precision == RAD_F32)
    k_loss<float><<<rows, 256, 0, ctx->stream>>>((const float *)I, (float *)dL, L, G.n[0], G.n[1], ctx->ang.n_ap,
                                                 ctx->ang.n_ang, G.f1, ctx->dang.dir, ctx->dang.dOmega);
  else
    k_loss<double><<<rows, 256, 0, ctx->stream>>>((const double *)I, (double *)dL, L, G.n[0], G.n[1],
                                                  ctx->ang.n_ap, ctx->ang.n_ang, G.f1, ctx->dang.dir,
                                                  ctx->dang.dOmega);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("loss launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

int launch_adjoint(rad_ctx *ctx, const void *, const rad_gas *, double, const rad_opts *, const void *, void *,
                   double *, double *, double *, std::string &err) {
  (void)ctx;
  err = "rad_step_adjoint is not built yet";
  return RAD_EUNSUPPORTED;
}

}  // namespace rad
