// Transposed transport of the adjoint, double, curved space with minimum-angle
// plane reconstruction of the angular face values (geodesic grids).
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<double, true, 2>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
