// Persistent batched kernel instantiations: the double-float solve (TSYLV_DF64), d = 4.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<dfl, 4, kFormLaplace>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 4, kFormLaplace>();
template int batched_occupancy_t<dfl, 4, kFormLaplace>();
template cudaError_t launch_batched_t<dfl, 4, kFormDTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 4, kFormDTerm>();
template int batched_occupancy_t<dfl, 4, kFormDTerm>();

}  // namespace tsylv
