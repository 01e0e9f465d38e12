// Fused refinement step instantiation, d = 4.
#include "fused_kernel.cuh"

namespace tsylv {

template cudaError_t launch_fused_t<4>(const FusedArgs&, int, cudaStream_t);
template cudaError_t prepare_fused_t<4>();
template int fused_occupancy_t<4>();
template cudaError_t launch_refine2_t<4>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<4>();

}  // namespace tsylv
