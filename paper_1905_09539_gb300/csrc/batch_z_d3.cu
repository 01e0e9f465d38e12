// Persistent kernel instantiations: complex FP64 (complex-triangular coefficients), d = 3.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<zd, 3, 0>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<zd, 3, 0>();
template int batched_occupancy_t<zd, 3, 0>();
template cudaError_t launch_batched_t<zd, 3, 1>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<zd, 3, 1>();
template int batched_occupancy_t<zd, 3, 1>();

}  // namespace tsylv
