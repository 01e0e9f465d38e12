// Wavefront kernel instantiations: element type double, d = 4.
#include "wave_kernel.cuh"

namespace tsylv {

template cudaError_t launch_wave_t<double, 4, false>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 4, false>();
template cudaError_t launch_wave_t<double, 4, true>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 4, true>();

}  // namespace tsylv
