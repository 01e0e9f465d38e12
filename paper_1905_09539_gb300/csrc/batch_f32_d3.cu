// Persistent batched kernel instantiations: element type float, d = 3.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<float, 3, false>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 3, false>();
template int batched_occupancy_t<float, 3, false>();
template cudaError_t launch_batched_t<float, 3, true>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 3, true>();
template int batched_occupancy_t<float, 3, true>();

}  // namespace tsylv
