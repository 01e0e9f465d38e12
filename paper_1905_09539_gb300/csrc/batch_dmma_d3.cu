// Persistent batched kernel instantiations: FP64 solve with FP64 DMMA tensor-core block updates, d = 3.
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<double, 3, false, kProdDMMA>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<double, 3, false, kProdDMMA>();
template int batched_occupancy_t<double, 3, false, kProdDMMA>();
template cudaError_t launch_batched_t<double, 3, true, kProdDMMA>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<double, 3, true, kProdDMMA>();
template int batched_occupancy_t<double, 3, true, kProdDMMA>();

}  // namespace tsylv
