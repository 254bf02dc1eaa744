// Moment contraction R^{AB} = sum_n I_n n^A n^B dOmega_n (Sec. 2.5), CUDA
// cores.  One warp per cell: lanes stride over the bins with ten running
// sums, a butterfly reduction combines the lanes, and lane 0 applies the
// FP64 frame change (coordinate frame e e R; fluid frame Lambda Lambda R
// with the boost of Sec. 2.1).
#include "rad_internal.h"

namespace rad {

// out^{ab} = L^a_A L^b_B R^{AB} for the ten components (00 01 02 03 11 12 13
// 22 23 33), written out with fixed indices.
__device__ __forceinline__ void frame_change(const double L[4][4], const double Rt[10], double out[10]) {
  const double R[4][4] = {{Rt[0], Rt[1], Rt[2], Rt[3]},
                          {Rt[1], Rt[4], Rt[5], Rt[6]},
                          {Rt[2], Rt[5], Rt[7], Rt[8]},
                          {Rt[3], Rt[6], Rt[8], Rt[9]}};
  double T[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int B = 0; B < 4; ++B) T[a][B] = L[a][0] * R[0][B] + L[a][1] * R[1][B] + L[a][2] * R[2][B] + L[a][3] * R[3][B];
  auto c = [&](int a, int b) { return T[a][0] * L[b][0] + T[a][1] * L[b][1] + T[a][2] * L[b][2] + T[a][3] * L[b][3]; };
  out[0] = c(0, 0);
  out[1] = c(0, 1);
  out[2] = c(0, 2);
  out[3] = c(0, 3);
  out[4] = c(1, 1);
  out[5] = c(1, 2);
  out[6] = c(1, 3);
  out[7] = c(2, 2);
  out[8] = c(2, 3);
  out[9] = c(3, 3);
}

// Boost Lambda^abar_Bhat to the fluid frame for tetrad-frame u^ihat (Sec. 2.1).
__device__ __forceinline__ void boost_matrix(double ux, double uy, double uz, double L[4][4]) {
  const double u[3] = {ux, uy, uz};
  const double u0 = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
  const double g = 1.0 / (1.0 + u0);
  L[0][0] = u0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    L[0][a + 1] = -u[a];
    L[a + 1][0] = -u[a];
#pragma unroll
    for (int b = 0; b < 3; ++b) L[a + 1][b + 1] = u[a] * u[b] * g + (a == b ? 1.0 : 0.0);
  }
}

template <typename R>
__global__ void k_moments_simt(const R *I, R *out, long long ncell, int ncol, int nap, int nang,
                               const double *dir, const double *dOmega, int frame, const ColGeo *cols,
                               const double *u) {
  long long cell = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (cell >= ncell) return;
  const R *row = I + cell * nap;
  R acc[10];
#pragma unroll
  for (int p = 0; p < 10; ++p) acc[p] = R(0);
  for (int n = lane; n < nang; n += 32) {
    R v = row[n] * (R)dOmega[n];
    R x = (R)dir[3 * n], y = (R)dir[3 * n + 1], z = (R)dir[3 * n + 2];
    R vx = v * x, vy = v * y, vz = v * z;
    acc[0] += v;
    acc[1] += vx;
    acc[2] += vy;
    acc[3] += vz;
    acc[4] += vx * x;
    acc[5] += vx * y;
    acc[6] += vx * z;
    acc[7] += vy * y;
    acc[8] += vy * z;
    acc[9] += vz * z;
  }
#pragma unroll
  for (int p = 0; p < 10; ++p)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], o);
  if (lane == 0) {
    double Rt[10], Ro[10];
    for (int p = 0; p < 10; ++p) Rt[p] = (double)acc[p];
    if (frame == RAD_FRAME_COORD) {
      double E[4][4];
      const ColGeo &cg = cols[cell % ncol];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int A = 0; A < 4; ++A) E[m][A] = cg.e[m][A];
      frame_change(E, Rt, Ro);
    } else if (frame == RAD_FRAME_FLUID) {
      double L[4][4];
      boost_matrix(u[3 * cell], u[3 * cell + 1], u[3 * cell + 2], L);
      frame_change(L, Rt, Ro);
    } else {
      for (int p = 0; p < 10; ++p) Ro[p] = Rt[p];
    }
    for (int p = 0; p < 10; ++p) out[cell * 10 + p] = (R)Ro[p];
  }
}

int launch_moments_bf16x3(rad_ctx *ctx, const float *I, int frame, const double *u, float *R,
                          cudaStream_t st, std::string &err);

int launch_moments(rad_ctx *ctx, const void *I, int precision, int frame, int method, const rad_gas *gas,
                   void *R, cudaStream_t st, std::string &err) {
  const DevGeom &G = ctx->geom;
  long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
  const double *u = (frame == RAD_FRAME_FLUID) ? gas->u : nullptr;
  if (method == RAD_MOM_BF16X3) return launch_moments_bf16x3(ctx, (const float *)I, frame, u, (float *)R, st, err);
  const int wpb = 8;
  unsigned blocks = (unsigned)((ncell + wpb - 1) / wpb);
  if (precision == RAD_F32)
    k_moments_simt<float><<<blocks, 32 * wpb, 0, st>>>(
        (const float *)I, (float *)R, ncell, G.n[0] * G.n[1], ctx->ang.n_ap, ctx->ang.n_ang, ctx->dang.dir,
        ctx->dang.dOmega, frame, G.cols, u);
  else
    k_moments_simt<double><<<blocks, 32 * wpb, 0, st>>>(
        (const double *)I, (double *)R, ncell, G.n[0] * G.n[1], ctx->ang.n_ap, ctx->ang.n_ang, ctx->dang.dir,
        ctx->dang.dOmega, frame, G.cols, u);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("moments launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
