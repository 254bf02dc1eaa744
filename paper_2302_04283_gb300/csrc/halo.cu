// Ghost exchange between blocks of a decomposed domain (the task list of
// Sec. 2: each stage's fluxes need the neighbouring blocks' cells next to
// the shared faces).  rad_halo_pack copies the kHaloLayers layers of an
// intensity array next to one face into a contiguous buffer, ordered by the
// distance from the face (layer 0 adjacent), which is the halo layout the
// stage kernel reads for the neighbouring block's opposite face:
//   x1 face: [layer][k][j][n_ap]   x2 face: [layer][k][i][n_ap]
//   x3 face: [layer][j][i][n_ap]
#include "rad_internal.h"

namespace rad {

namespace {

constexpr int kPackWarps = 4;

// One warp per row; rows are copied as 16-byte words (a padded row of n_ap
// elements is a multiple of 16 bytes in both precisions).
__global__ void __launch_bounds__(32 * kPackWarps) k_halo_pack(const uint4 *__restrict__ I, uint4 *__restrict__ buf,
                                                               int d, int side, int n1, int n2, int n3, int wpr,
                                                               long long nrows) {
  const long long row = (long long)blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  if (row >= nrows) return;
  const int lane = threadIdx.x & 31;
  const int B = d == 0 ? n2 : n1;
  const int A = d == 2 ? n2 : n3;
  const int b = (int)(row % B);
  const long long t = row / B;
  const int a = (int)(t % A);
  const int L = (int)(t / A);
  const int N = d == 0 ? n1 : (d == 1 ? n2 : n3);
  const int q = side ? N - 1 - L : L;
  size_t cell;
  if (d == 0) cell = ((size_t)a * n2 + b) * n1 + q;          // (k, j, i = q)
  else if (d == 1) cell = ((size_t)a * n2 + q) * n1 + b;     // (k, j = q, i)
  else cell = ((size_t)q * n2 + a) * n1 + b;                 // (k = q, j, i)
  const uint4 *src = I + cell * wpr;
  uint4 *dst = buf + (size_t)row * wpr;
  for (int w = lane; w < wpr; w += 32) dst[w] = __ldg(src + w);
}

}  // namespace

int launch_halo_pack(rad_ctx *ctx, const void *I, int precision, int dim, int side, void *buf, std::string &err) {
  const DevGeom &G = ctx->geom;
  const int esz = precision == RAD_F32 ? 4 : 8;
  const int wpr = ctx->ang.n_ap * esz / 16;
  const long long other = dim == 0 ? (long long)G.n[2] * G.n[1] : (dim == 1 ? (long long)G.n[2] * G.n[0]
                                                                            : (long long)G.n[1] * G.n[0]);
  const long long nrows = (long long)kHaloLayers * other;
  const long long blocks = (nrows + kPackWarps - 1) / kPackWarps;
  k_halo_pack<<<(unsigned)blocks, 32 * kPackWarps, 0, ctx->stream>>>((const uint4 *)I, (uint4 *)buf, dim, side,
                                                                    G.n[0], G.n[1], G.n[2], wpr, nrows);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("halo pack launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
