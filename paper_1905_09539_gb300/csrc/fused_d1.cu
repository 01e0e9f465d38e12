// Fused refinement step instantiation, d = 1.
#include "fused_kernel.cuh"

namespace tsylv {

template cudaError_t launch_fused_t<1>(const FusedArgs&, int, cudaStream_t);
template cudaError_t prepare_fused_t<1>();
template int fused_occupancy_t<1>();

}  // namespace tsylv
