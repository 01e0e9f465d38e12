// Persistent batched kernel instantiations: element type float, d = 2.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<float, 2, false>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 2, false>();
template int batched_occupancy_t<float, 2, false>();
template cudaError_t launch_batched_t<float, 2, true>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 2, true>();
template int batched_occupancy_t<float, 2, true>();

}  // namespace tsylv
