// Transposed transport of the adjoint, float, flat space.
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<float, false>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
