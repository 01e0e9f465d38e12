// Wavefront kernel instantiations for element type double.
#include "wave_kernel.cuh"

namespace tsylv {

template <>
cudaError_t launch_wave<double>(int d, bool generalized, int prod, const WaveArgs& a, cudaStream_t s) {
    (void)prod;
    return launch_wave_impl<double>(d, generalized, a, s);
}

template <>
cudaError_t prepare_wave<double>() {
    return prepare_wave_impl<double>();
}

}  // namespace tsylv
