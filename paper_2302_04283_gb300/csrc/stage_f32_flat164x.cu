// FP32 stage kernels without angular fluxes, level-4 row length fixed at
// compile time, with halo rows of faces shared with other blocks and the
// multigroup frequency divergence (the block path of the level-4 grid).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, false, 0, -kNapGeo4>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
