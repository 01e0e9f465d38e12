// Wavefront kernel instantiations: element type double, d = 2.
#include "wave_kernel.cuh"

namespace tsylv {

template cudaError_t launch_wave_t<double, 2, false>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 2, false>();
template cudaError_t launch_wave_t<double, 2, true>(const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave_t<double, 2, true>();

}  // namespace tsylv
