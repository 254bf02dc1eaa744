// Transposed transport of the adjoint, double, curved space with PLM angular
// reconstruction along the lines of a latitude-longitude grid.
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<double, true, 1>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
