// FP64 stage kernels with angular fluxes (curved space) and the
// minimum-angle plane reconstruction of the angular face values (geodesic grids).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<double, true, 2>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
