// Transposed transport of the adjoint, double, curved space (angular fluxes).
#include "adjoint_kernels.cuh"

namespace rad {

template cudaError_t launch_transport_adj<double, true>(const AdjArgs &A, cudaStream_t st);

}  // namespace rad
