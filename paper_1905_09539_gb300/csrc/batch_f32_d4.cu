// Persistent batched kernel instantiations: element type float, d = 4.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<float, 4, false>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 4, false>();
template int batched_occupancy_t<float, 4, false>();
template cudaError_t launch_batched_t<float, 4, true>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 4, true>();
template int batched_occupancy_t<float, 4, true>();

}  // namespace tsylv
