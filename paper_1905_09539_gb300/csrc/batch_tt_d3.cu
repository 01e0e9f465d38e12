// Persistent kernel instantiation: the paper's two-term form Eq. (3.1), FP64, d = 3.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<double, 3, kFormTwoTerm>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<double, 3, kFormTwoTerm>();
template int batched_occupancy_t<double, 3, kFormTwoTerm>();

}  // namespace tsylv
