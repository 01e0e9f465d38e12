// Persistent batched kernel instantiations: element type double, d = 5 (the Laplace form).
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<double, 5, false>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<double, 5, false>();
template int batched_occupancy_t<double, 5, false>();

}  // namespace tsylv
