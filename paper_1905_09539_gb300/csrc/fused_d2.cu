// Fused refinement step instantiation, d = 2.
#include "fused_kernel.cuh"

namespace tsylv {

template cudaError_t launch_fused_t<2>(const FusedArgs&, int, cudaStream_t);
template cudaError_t prepare_fused_t<2>();
template int fused_occupancy_t<2>();
template cudaError_t launch_refine2_t<2>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<2>();

}  // namespace tsylv
