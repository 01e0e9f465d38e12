// Persistent batched kernel instantiations: the paper's two-term form Eq. (3.1) in double-float
// arithmetic (TSYLV_DF64), d = 2, 3, 4.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<dfl, 2, kFormTwoTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 2, kFormTwoTerm>();
template int batched_occupancy_t<dfl, 2, kFormTwoTerm>();
template cudaError_t launch_batched_t<dfl, 3, kFormTwoTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 3, kFormTwoTerm>();
template int batched_occupancy_t<dfl, 3, kFormTwoTerm>();
template cudaError_t launch_batched_t<dfl, 4, kFormTwoTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<dfl, 4, kFormTwoTerm>();
template int batched_occupancy_t<dfl, 4, kFormTwoTerm>();

}  // namespace tsylv
