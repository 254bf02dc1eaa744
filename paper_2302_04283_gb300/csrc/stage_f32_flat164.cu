// FP32 stage kernels without angular fluxes (Cartesian Minkowski), specialised
// for the padded row of the level-4 geodesic grid (162 bins, 164 padded).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, false, 0, kNapGeo4>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
