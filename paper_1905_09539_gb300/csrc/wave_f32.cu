// Wavefront kernel instantiations for element type float.
#include "wave_kernel.cuh"

namespace tsylv {

template <>
cudaError_t launch_wave<float>(int d, bool generalized, int prod, const WaveArgs& a, cudaStream_t s) {
    (void)prod;
    return launch_wave_impl<float>(d, generalized, a, s);
}

template <>
cudaError_t prepare_wave<float>() {
    return prepare_wave_impl<float>();
}

}  // namespace tsylv
