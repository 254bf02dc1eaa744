// Transposed transport of the adjoint, double, flat space.
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<double, false>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
