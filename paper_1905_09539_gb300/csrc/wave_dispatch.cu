// Dispatch of the wavefront kernel over (element type, d, form).
#include "tsylv_internal.h"

namespace tsylv {

template <typename T, int D, int GEN>
cudaError_t launch_wave_t(const WaveArgs& a, cudaStream_t s);
template <typename T, int D, int GEN>
cudaError_t prepare_wave_t();

template <typename T>
cudaError_t launch_wave(int d, bool gen, int prod, const WaveArgs& a, cudaStream_t s) {
    (void)prod;
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return launch_wave_t<T, 1, false>(a, s);  // d = 1: both forms coincide
        case 4: return launch_wave_t<T, 2, false>(a, s);
        case 5: return launch_wave_t<T, 2, true>(a, s);
        case 6: return launch_wave_t<T, 3, false>(a, s);
        case 7: return launch_wave_t<T, 3, true>(a, s);
        case 8: return launch_wave_t<T, 4, false>(a, s);
        case 9: return launch_wave_t<T, 4, true>(a, s);
        case 10: return launch_wave_t<T, 5, false>(a, s);  // d = 5: the Laplace form only
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t prepare_wave() {
    cudaError_t e = cudaSuccess;
    if ((e = prepare_wave_t<T, 1, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 2, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 2, true>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 3, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 3, true>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 4, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 4, true>()) != cudaSuccess) return e;
    return prepare_wave_t<T, 5, false>();
}

template cudaError_t launch_wave<double>(int, bool, int, const WaveArgs&, cudaStream_t);
template cudaError_t launch_wave<float>(int, bool, int, const WaveArgs&, cudaStream_t);
template cudaError_t prepare_wave<double>();
template cudaError_t prepare_wave<float>();

}  // namespace tsylv
