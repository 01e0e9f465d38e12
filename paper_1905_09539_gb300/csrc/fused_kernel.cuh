// First two steps of the mixed-precision refinement of the Laplace form in
// one persistent launch (see Refine2Args): the second FP32 solve and both
// residuals follow the first solve block by block.
#pragma once

#include "apply_tile.cuh"
#include "batched.h"
#include "fused.h"
#include "wave_kernel.cuh"

namespace tsylv {

template <int D>
struct FusedCfg {
    using CW = WaveCfg<float, D, false>;
    using CA = apply_detail::ApplyCfg<D, kModeDF>;
    static constexpr size_t body = CW::smem > CA::smem ? CW::smem : CA::smem;
    static constexpr size_t oBarW = (body + 15) / 16 * 16;
    static constexpr size_t oBarA = oBarW + 8 * CW::NST;
    static constexpr size_t smem = oBarA + 8 * CA::NST;
};

template <int D, int PK>
__global__ void __launch_bounds__(kThreads) k_refine2(const Refine2Args f) {
    using F = FusedCfg<D>;
    using CW = typename F::CW;
    using CA = typename F::CA;
    constexpr int TD = CW::TD;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* barW = reinterpret_cast<uint64_t*>(smem_raw + F::oBarW);
    uint64_t* barA = reinterpret_cast<uint64_t*>(smem_raw + F::oBarA);
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        for (int q = 0; q < CW::NST; q++) dev::mbar_init(&barW[q], 1);
        for (int q = 0; q < CA::NST; q++) dev::mbar_init(&barA[q], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t usesW[CW::NST] = {};
    uint32_t usesA[CA::NST] = {};
    bool alive = true;  // false after a timed-out copy: no further copies on these barriers
    const WaveArgs& w1 = *f.w1;
    const WaveArgs& w2 = *f.w2;
    const float inv = static_cast<float>(1.0 / dev::step_scale(f.nrm[1]));
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(f.head, 1);
        __syncthreads();
        const int j = s_job;
        if (j >= f.njobs) break;
        const int code = f.jobs[j];
        const int kind = code >> 26;
        const long long t = code & ((1 << 26) - 1);
        // the job's own prerequisite (the sources of a solve are awaited inside it)
        const int* need = kind == 1 ? w1.ready + t : kind == 2 ? f.r1done + t : kind == 3 ? w2.ready + t : nullptr;
        if (need != nullptr && threadIdx.x == 0) {
            if (!dev::wait_at_least(need, 1, f.abort, f.timeout_ns)) atomicOr(w1.err, kErrTimeout);
            dev::fence_proxy_async_all();
        }
        __syncthreads();
        if (kind == 0 || kind == 2) {
            if (alive) alive = wave_tile<float, D, false, PK>(kind == 0 ? w1 : w2, t, 0, 1, usesW, barW);
            __syncthreads();
            if (threadIdx.x == 0) dev::publish(const_cast<int*>((kind == 0 ? w1 : w2).ready) + t, 1, nullptr);
        } else if (kind == 1) {
            if (alive) apply_detail::apply_tile<D, kModeDFh>(f.r1, t, smem_raw, barA, usesA);
            __syncthreads();
            // right-hand side of the second solve: R1 / s (exact scaling)
            const double* R = f.r1.R + t * TD;
            for (int e = threadIdx.x; e < TD; e += kThreads) f.X2[t * TD + e] = static_cast<float>(R[e]) * inv;
            __syncthreads();
            if (threadIdx.x == 0) dev::publish(f.r1done + t, 1, nullptr);
        } else {
            if (alive) apply_detail::apply_tile<D, kModeF32>(f.r2, t, smem_raw, barA, usesA);
            __syncthreads();
        }
    }
}

template <int D, int PK>
int refine2_occupancy_t() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refine2<D, PK>, kThreads, FusedCfg<D>::smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <int D, int PK>
cudaError_t launch_refine2_t(const Refine2Args& f, int grid, cudaStream_t s) {
    k_refine2<D, PK><<<grid, kThreads, FusedCfg<D>::smem, s>>>(f);
    return cudaGetLastError();
}

template <int D, int PK>
cudaError_t prepare_refine2_t() {
    return cudaFuncSetAttribute(k_refine2<D, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(FusedCfg<D>::smem));
}

}  // namespace tsylv
