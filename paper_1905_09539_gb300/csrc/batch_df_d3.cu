// Persistent batched kernel instantiations: the double-float solve (TSYLV_DF64), d = 3.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<dfl, 3, kFormLaplace>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 3, kFormLaplace>();
template int batched_occupancy_t<dfl, 3, kFormLaplace>();
template cudaError_t launch_batched_t<dfl, 3, kFormDTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 3, kFormDTerm>();
template int batched_occupancy_t<dfl, 3, kFormDTerm>();

}  // namespace tsylv
