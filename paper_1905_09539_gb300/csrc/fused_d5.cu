// Pipelined refinement launch instantiations, d = 5 (native, TF32 and BF16 block updates).
#include "fused_kernel.cuh"

namespace tsylv {

template cudaError_t launch_refine2_t<5, kProdNative>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<5, kProdNative>();
template cudaError_t prepare_refine2_t<5, kProdNative>();
template cudaError_t launch_refine2_t<5, kProdTF32>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<5, kProdTF32>();
template cudaError_t prepare_refine2_t<5, kProdTF32>();
template cudaError_t launch_refine2_t<5, kProdBF16>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<5, kProdBF16>();
template cudaError_t prepare_refine2_t<5, kProdBF16>();

}  // namespace tsylv
