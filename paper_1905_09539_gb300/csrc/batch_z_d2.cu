// Persistent kernel instantiations: complex FP64 (complex-triangular coefficients), d = 2.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<zd, 2, 0>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<zd, 2, 0>();
template int batched_occupancy_t<zd, 2, 0>();
template cudaError_t launch_batched_t<zd, 2, 1>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<zd, 2, 1>();
template int batched_occupancy_t<zd, 2, 1>();

}  // namespace tsylv
