// FP32 stage kernels with angular fluxes (curved metrics, spherical tetrads).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, true>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
