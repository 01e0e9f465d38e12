// Wavefront kernel instantiations: element type float, d = 5 (the Laplace form).
#include "wave_kernel.cuh"

namespace tsylv {

template cudaError_t launch_wave_t<float, 5, false>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<float, 5, false>();

}  // namespace tsylv
