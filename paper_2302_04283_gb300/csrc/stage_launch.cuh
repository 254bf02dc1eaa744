// Launch of the stage kernel for one precision and geometry class: picks the
// compile-time variant (donor cell, PLM or PPM, stage 1 or 2, with or without
// the optical-depth flux weighting).  Included by the stage_*.cu translation
// units only, each of which instantiates one (precision, geometry) pair.
#pragma once

#include "step_kernel.cuh"

namespace rad {

template <typename R, bool ANG, int RC, bool ST2, bool TAU, int AR, int NAP>
cudaError_t launch_stage_t(const StageArgs &a, int threads, dim3 grid, cudaStream_t st) {
  size_t smem = stage_smem<R, ANG>(threads, a.nap, a.kc, a.depth, TAU, stage_rows(RC), AR == 2);
  auto kern = k_stage<R, ANG, RC, ST2, TAU, AR, NAP>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // the kernel keeps its working set in shared memory: prefer the largest carve-out
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  kern<<<grid, threads + 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename R, bool ANG, bool TAU, int AR, int NAP>
cudaError_t launch_stage_pt(const StageArgs &a, int threads, dim3 grid, cudaStream_t st) {
  if (a.recon == RAD_RECON_PPM)
    return a.stage2 ? launch_stage_t<R, ANG, RAD_RECON_PPM, true, TAU, AR, NAP>(a, threads, grid, st)
                    : launch_stage_t<R, ANG, RAD_RECON_PPM, false, TAU, AR, NAP>(a, threads, grid, st);
  if (a.recon == RAD_RECON_PLM)
    return a.stage2 ? launch_stage_t<R, ANG, RAD_RECON_PLM, true, TAU, AR, NAP>(a, threads, grid, st)
                    : launch_stage_t<R, ANG, RAD_RECON_PLM, false, TAU, AR, NAP>(a, threads, grid, st);
  return a.stage2 ? launch_stage_t<R, ANG, RAD_RECON_DC, true, TAU, AR, NAP>(a, threads, grid, st)
                  : launch_stage_t<R, ANG, RAD_RECON_DC, false, TAU, AR, NAP>(a, threads, grid, st);
}

template <typename R, bool ANG, int AR, int NAP>
cudaError_t launch_stage_rp(const StageArgs &a, cudaStream_t st) {
  if (NAP != 0 && a.nap != (NAP > 0 ? NAP : -NAP)) return cudaErrorInvalidValue;
  const int threads = (a.nap / 2 + 31) / 32 * 32;     // two bins per consumer thread
  const int nchunk = (a.n3 + a.kc - 1) / a.kc;
  const dim3 grid((unsigned)((long long)a.n1 * a.n2 * nchunk));
  return a.tau_const > 0.0 ? launch_stage_pt<R, ANG, true, AR, NAP>(a, threads, grid, st)
                           : launch_stage_pt<R, ANG, false, AR, NAP>(a, threads, grid, st);
}

}  // namespace rad
