// Persistent kernel instantiations: complex FP64 (complex-triangular coefficients), d = 1.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<zd, 1, 0>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<zd, 1, 0>();
template int batched_occupancy_t<zd, 1, 0>();

}  // namespace tsylv
