// FP32 stage kernels with angular fluxes (curved space) and the
// minimum-angle plane reconstruction of the angular face values (geodesic grids).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, true, 2>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
