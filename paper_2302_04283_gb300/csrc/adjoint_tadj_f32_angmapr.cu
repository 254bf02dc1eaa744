// Transposed transport of the adjoint, float, curved space with minimum-angle
// plane reconstruction of the angular face values (geodesic grids).
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<float, true, 2>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
