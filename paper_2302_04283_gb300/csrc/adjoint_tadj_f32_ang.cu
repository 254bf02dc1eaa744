// Transposed transport of the adjoint, float, curved space (angular fluxes).
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<float, true>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
