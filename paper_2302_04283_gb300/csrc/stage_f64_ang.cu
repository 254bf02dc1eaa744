// FP64 stage kernels with angular fluxes (curved metrics, spherical tetrads).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<double, true>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
