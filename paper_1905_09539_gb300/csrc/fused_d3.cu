// Fused refinement step instantiation, d = 3.
#include "fused_kernel.cuh"

namespace tsylv {

template cudaError_t launch_fused_t<3>(const FusedArgs&, int, cudaStream_t);
template cudaError_t prepare_fused_t<3>();
template int fused_occupancy_t<3>();
template cudaError_t launch_refine2_t<3>(const Refine2Args&, int, cudaStream_t);
template int refine2_occupancy_t<3>();

}  // namespace tsylv
