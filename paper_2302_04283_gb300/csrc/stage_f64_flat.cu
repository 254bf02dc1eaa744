// FP64 stage kernels without angular fluxes (Cartesian Minkowski).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<double, false>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
