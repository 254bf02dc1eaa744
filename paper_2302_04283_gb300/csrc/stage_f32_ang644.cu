// FP32 stage kernels with angular fluxes (curved space), specialised for the
// padded row of the level-8 geodesic grid (642 bins, 644 padded).
#include "stage_launch.cuh"

namespace rad {

template cudaError_t launch_stage_rp<float, true, 0, kNapGeo8>(const StageArgs &a, cudaStream_t st);

}  // namespace rad
