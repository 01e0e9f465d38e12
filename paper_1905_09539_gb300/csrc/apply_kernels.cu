// Operator application kernels (residual of the refinement): FP64, DF64
// (float pairs on the FP32 pipes), DF64 on a float source (the first
// refinement step, whose iterate is a scaled FP32 solution) and plain FP32
// (the residual update of a refinement step from its FP32 correction).
#include "apply_kernel.cuh"
#include "device_common.cuh"

#include "apply_tile.cuh"

namespace tsylv {

namespace {

using namespace apply_detail;

template <int D, int MD>
__device__ __forceinline__ void init_apply_barriers(unsigned char* smem) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + ApplyCfg<D, MD>::oBar);
    if (threadIdx.x == 0) {
        for (int q = 0; q < ApplyCfg<D, MD>::NST; q++) dev::mbar_init(&bar[q], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
}

template <int D, int MD>
__global__ void __launch_bounds__(kThreads) k_apply(const ApplyArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (static_cast<long long>(blockIdx.x) >= a.ntiles) return;
    init_apply_barriers<D, MD>(smem);
    apply_tile<D, MD>(a, blockIdx.x, smem, reinterpret_cast<uint64_t*>(smem + ApplyCfg<D, MD>::oBar), nullptr);
}

// Many independent applies in one launch: CTA b runs block jobs[b].y of the
// apply eqs[jobs[b].x] (every CTA owns one block, as in k_apply).
template <int D, int MD>
__global__ void __launch_bounds__(kThreads) k_apply_batched(const ApplyArgs* __restrict__ eqs,
                                                            const int2* __restrict__ jobs, int njobs) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (static_cast<int>(blockIdx.x) >= njobs) return;
    const int2 jb = jobs[blockIdx.x];
    init_apply_barriers<D, MD>(smem);
    apply_tile<D, MD>(eqs[jb.x], jb.y, smem, reinterpret_cast<uint64_t*>(smem + ApplyCfg<D, MD>::oBar), nullptr);
}

template <int D, int MD>
cudaError_t launch_apply_t(const ApplyArgs& a, cudaStream_t s) {
    using C = ApplyCfg<D, MD>;
    k_apply<D, MD><<<static_cast<unsigned>(a.ntiles), kThreads, C::smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int MD>
cudaError_t prepare_apply_t() {
    return cudaFuncSetAttribute(k_apply<D, MD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(ApplyCfg<D, MD>::smem));
}

template <int D, int MD>
cudaError_t launch_apply_batched_t(const ApplyArgs* eqs, const int2* jobs, int njobs, cudaStream_t s) {
    using C = ApplyCfg<D, MD>;
    if (njobs <= 0) return cudaSuccess;
    k_apply_batched<D, MD><<<static_cast<unsigned>(njobs), kThreads, C::smem, s>>>(eqs, jobs, njobs);
    return cudaGetLastError();
}

template <int D, int MD>
cudaError_t prepare_apply_batched_t() {
    return cudaFuncSetAttribute(k_apply_batched<D, MD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(ApplyCfg<D, MD>::smem));
}

template <int MD>
cudaError_t launch_apply_m(int d, const ApplyArgs& a, cudaStream_t s) {
    switch (d) {
        case 1: return launch_apply_t<1, MD>(a, s);
        case 2: return launch_apply_t<2, MD>(a, s);
        case 3: return launch_apply_t<3, MD>(a, s);
        case 4: return launch_apply_t<4, MD>(a, s);
        case 5: return launch_apply_t<5, MD>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int MD>
cudaError_t prepare_apply_m() {
    cudaError_t e;
    if ((e = prepare_apply_t<1, MD>()) != cudaSuccess) return e;
    if ((e = prepare_apply_t<2, MD>()) != cudaSuccess) return e;
    if ((e = prepare_apply_t<3, MD>()) != cudaSuccess) return e;
    if ((e = prepare_apply_t<4, MD>()) != cudaSuccess) return e;
    return prepare_apply_t<5, MD>();
}

}  // namespace

template <bool DF>
cudaError_t launch_apply(int d, const ApplyArgs& a, cudaStream_t s) {
    return launch_apply_m<DF ? kModeDF : kModeF64>(d, a, s);
}

template <bool DF>
cudaError_t prepare_apply() {
    return prepare_apply_m<DF ? kModeDF : kModeF64>();
}

cudaError_t launch_apply_f32(int d, const ApplyArgs& a, cudaStream_t s) { return launch_apply_m<kModeF32>(d, a, s); }
cudaError_t prepare_apply_f32() { return prepare_apply_m<kModeF32>(); }

cudaError_t launch_apply_dfh(int d, const ApplyArgs& a, cudaStream_t s) { return launch_apply_m<kModeDFh>(d, a, s); }
cudaError_t prepare_apply_dfh() { return prepare_apply_m<kModeDFh>(); }

cudaError_t launch_apply_batched(int d, int mode, const ApplyArgs* eqs, const int2* jobs, int njobs, cudaStream_t s) {
#define TSYLV_APPLY_B(DD)                                                                          \
    if (d == DD) {                                                                                 \
        if (mode == kModeF64) return launch_apply_batched_t<DD, kModeF64>(eqs, jobs, njobs, s);   \
        if (mode == kModeDF) return launch_apply_batched_t<DD, kModeDF>(eqs, jobs, njobs, s);     \
        if (mode == kModeF32) return launch_apply_batched_t<DD, kModeF32>(eqs, jobs, njobs, s);   \
        if (mode == kModeDFh) return launch_apply_batched_t<DD, kModeDFh>(eqs, jobs, njobs, s);   \
    }
    TSYLV_APPLY_B(1)
    TSYLV_APPLY_B(2)
    TSYLV_APPLY_B(3)
    TSYLV_APPLY_B(4)
    TSYLV_APPLY_B(5)
#undef TSYLV_APPLY_B
    return cudaErrorInvalidValue;
}

cudaError_t prepare_apply_batched() {
    cudaError_t e = cudaSuccess;
#define TSYLV_PREP_B(DD)                                                                              \
    if (e == cudaSuccess) e = prepare_apply_batched_t<DD, kModeF64>();                                \
    if (e == cudaSuccess) e = prepare_apply_batched_t<DD, kModeDF>();                                 \
    if (e == cudaSuccess) e = prepare_apply_batched_t<DD, kModeF32>();                                \
    if (e == cudaSuccess) e = prepare_apply_batched_t<DD, kModeDFh>();
    TSYLV_PREP_B(1)
    TSYLV_PREP_B(2)
    TSYLV_PREP_B(3)
    TSYLV_PREP_B(4)
    TSYLV_PREP_B(5)
#undef TSYLV_PREP_B
    return e;
}

template cudaError_t launch_apply<false>(int, const ApplyArgs&, cudaStream_t);
template cudaError_t launch_apply<true>(int, const ApplyArgs&, cudaStream_t);
template cudaError_t prepare_apply<false>();
template cudaError_t prepare_apply<true>();

}  // namespace tsylv
