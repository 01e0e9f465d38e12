// Dispatch of the pipelined refinement launch over d and the product kind.
#include "fused.h"

namespace tsylv {

template <int D, int PK>
cudaError_t launch_refine2_t(const Refine2Args& f, int grid, cudaStream_t s);
template <int D, int PK>
int refine2_occupancy_t();
template <int D, int PK>
cudaError_t prepare_refine2_t();

namespace {

template <int PK>
cudaError_t launch_pk(int d, const Refine2Args& f, int grid, cudaStream_t s) {
    switch (d) {  // d = 1 is not offered: the single-mode solve keeps separate launches
        case 2: return launch_refine2_t<2, PK>(f, grid, s);
        case 3: return launch_refine2_t<3, PK>(f, grid, s);
        case 4: return launch_refine2_t<4, PK>(f, grid, s);
        case 5: return launch_refine2_t<5, PK>(f, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int PK>
int occupancy_pk(int d) {
    switch (d) {
        case 2: return refine2_occupancy_t<2, PK>();
        case 3: return refine2_occupancy_t<3, PK>();
        case 4: return refine2_occupancy_t<4, PK>();
        case 5: return refine2_occupancy_t<5, PK>();
        default: return 1;
    }
}

template <int PK>
cudaError_t prepare_pk() {
    cudaError_t e;
    if ((e = prepare_refine2_t<2, PK>()) != cudaSuccess) return e;
    if ((e = prepare_refine2_t<3, PK>()) != cudaSuccess) return e;
    if ((e = prepare_refine2_t<4, PK>()) != cudaSuccess) return e;
    return prepare_refine2_t<5, PK>();
}

}  // namespace

cudaError_t launch_refine2(int d, int prod, const Refine2Args& f, int grid, cudaStream_t s) {
    switch (prod) {
        case kProdNative: return launch_pk<kProdNative>(d, f, grid, s);
        case kProdTF32: return launch_pk<kProdTF32>(d, f, grid, s);
        case kProdBF16: return launch_pk<kProdBF16>(d, f, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int refine2_occupancy(int d, int prod) {
    switch (prod) {
        case kProdTF32: return occupancy_pk<kProdTF32>(d);
        case kProdBF16: return occupancy_pk<kProdBF16>(d);
        default: return occupancy_pk<kProdNative>(d);
    }
}

cudaError_t prepare_refine2() {
    cudaError_t e = prepare_pk<kProdNative>();
    if (e == cudaSuccess) e = prepare_pk<kProdTF32>();
    if (e == cudaSuccess) e = prepare_pk<kProdBF16>();
    return e;
}

}  // namespace tsylv
