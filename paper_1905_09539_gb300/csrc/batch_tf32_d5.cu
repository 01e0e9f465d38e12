// Persistent batched kernel instantiations: FP32 solve with TF32 tensor-core block updates, d = 5 (the Laplace form).
#include "batched_kernel.cuh"

namespace tsylv {

template cudaError_t launch_batched_t<float, 5, false, kProdTF32>(const BatchArgs&, int, cudaStream_t);
template cudaError_t prepare_batched_t<float, 5, false, kProdTF32>();
template int batched_occupancy_t<float, 5, false, kProdTF32>();

}  // namespace tsylv
