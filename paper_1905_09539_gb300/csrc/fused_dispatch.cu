// Dispatch of the fused refinement step over d.
#include "fused.h"
#include "fused_kernel.cuh"

namespace tsylv {

template <int D>
cudaError_t launch_fused_t(const FusedArgs& f, int grid, cudaStream_t s);
template <int D>
cudaError_t prepare_fused_t();
template <int D>
int fused_occupancy_t();

cudaError_t launch_fused(int d, const FusedArgs& f, int grid, cudaStream_t s) {
    switch (d) {
        case 1: return launch_fused_t<1>(f, grid, s);
        case 2: return launch_fused_t<2>(f, grid, s);
        case 3: return launch_fused_t<3>(f, grid, s);
        case 4: return launch_fused_t<4>(f, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_fused() {
    cudaError_t e;
    if ((e = prepare_fused_t<1>()) != cudaSuccess) return e;
    if ((e = prepare_fused_t<2>()) != cudaSuccess) return e;
    if ((e = prepare_fused_t<3>()) != cudaSuccess) return e;
    return prepare_fused_t<4>();
}

template <int D>
cudaError_t launch_refine2_t(const Refine2Args& f, int grid, cudaStream_t s);
template <int D>
int refine2_occupancy_t();

cudaError_t launch_refine2(int d, const Refine2Args& f, int grid, cudaStream_t s) {
    switch (d) {  // d = 1 is not offered (its fused launch is refused, see the fused first step)
        case 2: return launch_refine2_t<2>(f, grid, s);
        case 3: return launch_refine2_t<3>(f, grid, s);
        case 4: return launch_refine2_t<4>(f, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int refine2_occupancy(int d) {
    switch (d) {
        case 2: return refine2_occupancy_t<2>();
        case 3: return refine2_occupancy_t<3>();
        case 4: return refine2_occupancy_t<4>();
        default: return 1;
    }
}

int fused_occupancy(int d) {
    switch (d) {
        case 1: return fused_occupancy_t<1>();
        case 2: return fused_occupancy_t<2>();
        case 3: return fused_occupancy_t<3>();
        case 4: return fused_occupancy_t<4>();
        default: return 1;
    }
}

}  // namespace tsylv
