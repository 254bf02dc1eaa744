// Moment contraction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// R^{AB} = sum_n I_n n^A n^B dOmega_n is the product D[cells x 16] =
// I[cells x K] . W^T[16 x K] with W[n][p] = n^A n^B dOmega_n for the ten
// pairs p (columns 10..15 zero, bins >= n_ang zero).  To keep FP32 accuracy
// on bf16 tensor cores both operands are split, x = hi + lo with hi =
// bf16(x), lo = bf16(x - hi), and D accumulates hi.hi + hi.lo + lo.hi in
// FP32 (the lo.lo term is below 2^-16 relative).
//
// One CTA of 128 threads owns a tile of 128 cells (M = 128, one TMEM lane per
// cell) and walks K in chunks of 64 bins: every thread converts its share of
// the FP32 rows into bf16 hi/lo and stores them in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix); one thread issues
// 4 x 3 tcgen05.mma (M=128, N=16, K=16) into a TMEM accumulator and commits
// to an mbarrier; after the last chunk each warp reads its 32 lanes back
// with tcgen05.ld and writes the 10 components.  W^T hi/lo is built once on
// the host and copied into shared memory per CTA.  Every wait is bounded: on
// timeout the CTA records an error, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rad_internal.h"

namespace rad {

constexpr int kTcM = 128;           // cells per tile
constexpr int kTcN = 16;            // moment columns (10 used)
constexpr int kTcKC = 64;           // bins per K chunk
constexpr int kTcThreads = 128;
constexpr int kTcErrTimeout = 1 << 3;  // reported as RAD_ECUDA by rad_check
constexpr long long kTcSpinLimit = 1ll << 24;

// byte offsets of the K-major no-swizzle layouts
//   A (128 x 64 chunk): core (mg, kg) at (kg * 16 + mg) * 128  -> SBO 128, LBO 2048
//   B (16 x Kp):        core (ng, kg) at (kg * 2 + ng) * 128   -> SBO 128, LBO 256
constexpr uint32_t kALbo = 2048, kASbo = 128, kBLbo = 256, kBSbo = 128;
constexpr uint32_t kATile = kTcM * kTcKC * 2;   // 16 KB per operand half

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: D f32, A bf16, B bf16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (long long it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 0) {                       // bounded in time as well as in polls
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (it == 0) t0 = now;
      else if (now - t0 > 2000000000ull) return false;
    }
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  uint32_t r;
  memcpy(&r, &v, 4);
  return r;
}

__global__ void __launch_bounds__(kTcThreads) k_moments_tc(const float *__restrict__ I, float *__restrict__ out,
                                                         long long ncell, int nap, int nang, int kp,
                                                         const uint4 *__restrict__ wt, int frame,
                                                         const ColGeoF *cols, int ncol, const double *u,
                                                         int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *Ah = sm;                    // [kATile]
  unsigned char *Al = sm + kATile;           // [kATile]
  unsigned char *Bw = sm + 2 * kATile;       // hi then lo, kp * 16 * 2 bytes each
  const uint32_t bbytes = (uint32_t)kp * kTcN * 2;
  uint64_t *bar = (uint64_t *)(Bw + 2 * bbytes);
  uint32_t *tslot = (uint32_t *)(bar + 1);
  const int t = threadIdx.x, warp = t >> 5;

  // W^T hi / lo (prebuilt layout) into shared memory
  const int nvec = (int)(2 * bbytes / 16);
  for (int v = t; v < nvec; v += kTcThreads) ((uint4 *)Bw)[v] = wt[v];
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t sAh = smem_addr(Ah), sAl = smem_addr(Al), sBh = smem_addr(Bw), sBl = smem_addr(Bw + bbytes);
  uint32_t phase = 0;
  bool failed = false;

  const long long ntile = (ncell + kTcM - 1) / kTcM;
  constexpr int kSeg = (kTcM * kTcKC / 8) / kTcThreads;   // 8-bin segments per thread and chunk
  // segment s of a chunk: cell m of the tile, bins kseg * 8 .. + 7 of the chunk
  auto seg_m = [&](int it) { const int s = it * kTcThreads + t, g = s >> 5; return (g >> 1) * 8 + ((s & 31) >> 2); };
  auto seg_k = [&](int it) { const int s = it * kTcThreads + t, g = s >> 5; return (g & 1) * 4 + (s & 3); };
  // global loads of one chunk into registers (zeros outside the grid and the bins)
  float4 v[2 * kSeg];
  auto load = [&](long long tile, int k0) {
#pragma unroll
    for (int it = 0; it < kSeg; ++it) {
      const long long cell = tile * kTcM + seg_m(it);
      const int k = k0 + seg_k(it) * 8;
      const float *row = I + cell * nap;
      v[2 * it] = (cell < ncell && k < nap) ? __ldg((const float4 *)(row + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[2 * it + 1] = (cell < ncell && k + 4 < nap) ? __ldg((const float4 *)(row + k + 4))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  // split into bf16 hi / lo in the K-major core-matrix layout
  auto convert = [&](int k0) {
#pragma unroll
    for (int it = 0; it < kSeg; ++it) {
      const int m = seg_m(it), kseg = seg_k(it), k = k0 + kseg * 8;
      float x[8] = {v[2 * it].x, v[2 * it].y, v[2 * it].z, v[2 * it].w,
                    v[2 * it + 1].x, v[2 * it + 1].y, v[2 * it + 1].z, v[2 * it + 1].w};
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (k + e >= nang) x[e] = 0.0f;                 // padding bins are not data
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * e]), h1 = __float2bfloat16_rn(x[2 * e + 1]);
        float r0 = x[2 * e] - __bfloat162float(h0), r1 = x[2 * e + 1] - __bfloat162float(h1);
        __nv_bfloat162 hh;
        hh.x = h0;
        hh.y = h1;
        memcpy(&h[e], &hh, 4);
        l[e] = pack_bf16(r0, r1);
      }
      const uint32_t off = (uint32_t)(kseg * 16 + (m >> 3)) * 128u + (uint32_t)(m & 7) * 16u;
      *(uint4 *)(Ah + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *(uint4 *)(Al + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  };

  // software pipeline over (tile, chunk) units: the loads of the next unit are
  // in flight while the tensor cores work on the current one
  long long tile = blockIdx.x;
  int k0 = 0;
  if (tile < ntile) load(tile, k0);
  while (tile < ntile && !failed) {
    convert(k0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTcKC / 16; ++kk) {
        const uint32_t kb = (uint32_t)((k0 / 16 + kk) * 2) * kBLbo;   // 2 core matrices per K step
        const uint64_t ah = umma_desc(sAh + kk * 2 * kALbo, kALbo, kASbo);
        const uint64_t al = umma_desc(sAl + kk * 2 * kALbo, kALbo, kASbo);
        const uint64_t bh = umma_desc(sBh + kb, kBLbo, kBSbo);
        const uint64_t bl = umma_desc(sBl + kb, kBLbo, kBSbo);
        const uint32_t first = (k0 == 0 && kk == 0) ? 0u : 1u;
        mma_bf16(tmem, ah, bh, first);
        mma_bf16(tmem, ah, bl, 1u);
        mma_bf16(tmem, al, bh, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(bar))
                   : "memory");
    }
    // next unit's loads, then wait for the MMAs (they read shared memory)
    const long long cur_tile = tile;
    const int cur_k0 = k0;
    k0 += kTcKC;
    if (k0 >= kp) {
      k0 = 0;
      tile += gridDim.x;
    }
    if (tile < ntile) load(tile, k0);
    const bool ok = mbar_wait(smem_addr(bar), phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {   // the decision is uniform across the CTA
      if (t == 0) atomicOr(err, kTcErrTimeout);
      failed = true;
      break;
    }
    if (cur_k0 + kTcKC < kp) continue;     // the tile has more chunks
    const long long cell0 = cur_tile * kTcM;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: lane m of TMEM holds the 16 sums of cell cell0 + m
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const long long cell = cell0 + t;
    if (cell < ncell) {
      float Rt[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) Rt[p] = __uint_as_float(r[p]);
      float Ro[10];
      if (frame == RAD_FRAME_TETRAD) {
#pragma unroll
        for (int p = 0; p < 10; ++p) Ro[p] = Rt[p];
      } else {
        float L[4][4];
        if (frame == RAD_FRAME_COORD) {
          const ColGeoF &cg = cols[cell % ncol];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) L[a][b] = cg.e[a][b];
        } else {
          const float ux = (float)u[3 * cell], uy = (float)u[3 * cell + 1], uz = (float)u[3 * cell + 2];
          const float uu[3] = {ux, uy, uz};
          const float u0 = sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
          L[0][0] = u0;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            L[0][a + 1] = -uu[a];
            L[a + 1][0] = -uu[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) L[a + 1][b + 1] = uu[a] * uu[b] / (1.0f + u0) + (a == b ? 1.0f : 0.0f);
          }
        }
        const float R4[4][4] = {{Rt[0], Rt[1], Rt[2], Rt[3]},
                                {Rt[1], Rt[4], Rt[5], Rt[6]},
                                {Rt[2], Rt[5], Rt[7], Rt[8]},
                                {Rt[3], Rt[6], Rt[8], Rt[9]}};
        float T4[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int B = 0; B < 4; ++B)
            T4[a][B] = L[a][0] * R4[0][B] + L[a][1] * R4[1][B] + L[a][2] * R4[2][B] + L[a][3] * R4[3][B];
        const int pa[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3}, pb[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
#pragma unroll
        for (int p = 0; p < 10; ++p)
          Ro[p] = T4[pa[p]][0] * L[pb[p]][0] + T4[pa[p]][1] * L[pb[p]][1] + T4[pa[p]][2] * L[pb[p]][2] +
                  T4[pa[p]][3] * L[pb[p]][3];
      }
      float *o = out + cell * 10;
#pragma unroll
      for (int p = 0; p < 10; ++p) o[p] = Ro[p];
    }
    // all lanes have read TMEM before the next tile's first MMA overwrites it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

namespace {

uint16_t bf16_bits(float x) {
  // round to nearest even (finite inputs)
  uint32_t b;
  std::memcpy(&b, &x, 4);
  uint32_t rnd = 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)((b + rnd) >> 16);
}
float bf16_to_float(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

}  // namespace

// Build W^T = (n^A n^B dOmega)^T split into bf16 hi / lo in the B layout.
static int build_wt(rad_ctx *ctx, int kp, std::string &err) {
  const AngleGrid &g = ctx->ang;
  const int pa[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3}, pb[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
  size_t half = (size_t)kp * kTcN;          // bf16 elements per operand half
  std::vector<uint16_t> buf(2 * half, 0);
  for (int n = 0; n < g.n_ang; ++n) {
    double nv[4] = {1.0, g.dir[3 * n], g.dir[3 * n + 1], g.dir[3 * n + 2]};
    for (int p = 0; p < 10; ++p) {
      float w = (float)(nv[pa[p]] * nv[pb[p]] * g.dOmega[n]);
      uint16_t hi = bf16_bits(w);
      uint16_t lo = bf16_bits(w - bf16_to_float(hi));
      // element (row p, k = n): core (p / 8, n / 8), row p % 8, column n % 8
      size_t off = ((size_t)(n / 8) * 2 + p / 8) * 64 + (p % 8) * 8 + (n % 8);
      buf[off] = hi;
      buf[half + off] = lo;
    }
  }
  cudaFree(ctx->wt_dev);
  ctx->wt_dev = nullptr;
  if (cudaMalloc(&ctx->wt_dev, buf.size() * 2) != cudaSuccess) {
    err = "moment weight allocation failed";
    return RAD_ENOMEM;
  }
  cudaMemcpyAsync(ctx->wt_dev, buf.data(), buf.size() * 2, cudaMemcpyHostToDevice, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  ctx->wt_kp = kp;
  ctx->wt_level = g.level;
  return RAD_OK;
}

int launch_moments_bf16x3(rad_ctx *ctx, const float *I, int frame, const double *u, float *R, cudaStream_t st,
                          std::string &err) {
  const DevGeom &G = ctx->geom;
  const int kp = (ctx->ang.n_ap + kTcKC - 1) / kTcKC * kTcKC;
  if (ctx->wt_dev == nullptr || ctx->wt_kp != kp || ctx->wt_level != ctx->ang.level) {
    int st = build_wt(ctx, kp, err);
    if (st != RAD_OK) return st;
  }
  const long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
  // operands (hi, lo) + W^T (hi, lo) + barrier and TMEM slot
  size_t smem = 2 * (size_t)kATile + 2 * (size_t)kp * kTcN * 2 + 64;
  smem = (smem + 1023) / 1024 * 1024;
  if (smem > 200 * 1024) {
    err = "split-bf16 moments: too many bins for shared memory";
    return RAD_EUNSUPPORTED;
  }
  cudaError_t ce = cudaFuncSetAttribute(k_moments_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce != cudaSuccess) {
    err = std::string("split-bf16 moments: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long ntile = (ncell + kTcM - 1) / kTcM;
  // four resident CTAs per SM keep enough loads in flight for HBM
  long long blocks = std::min<long long>(ntile, (long long)nsm * 4);
  k_moments_tc<<<(unsigned)blocks, kTcThreads, smem, st>>>(I, R, ncell, ctx->ang.n_ap, ctx->ang.n_ang, kp,
                                                                     (const uint4 *)ctx->wt_dev, frame, G.colsF,
                                                                     G.n[0] * G.n[1], u, ctx->err_word);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("split-bf16 moments launch failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  return RAD_OK;
}

}  // namespace rad
