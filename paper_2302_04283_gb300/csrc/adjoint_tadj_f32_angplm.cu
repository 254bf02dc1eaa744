// Transposed transport of the adjoint, float, curved space with PLM angular
// reconstruction along the lines of a latitude-longitude grid.
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<float, true, 1>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
