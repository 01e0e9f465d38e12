// Wavefront kernel instantiations: element type double, d = 3.
#include "wave_kernel.cuh"

namespace tsylv {

template cudaError_t launch_wave_t<double, 3, false>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 3, false>();
template cudaError_t launch_wave_t<double, 3, true>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 3, true>();

}  // namespace tsylv
