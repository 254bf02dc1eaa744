// F32 stage kernels with angular fluxes and PLM angular reconstruction
// along the lines of a latitude-longitude grid.
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, true, 1>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
