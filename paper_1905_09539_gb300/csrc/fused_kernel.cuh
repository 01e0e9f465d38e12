// First step of the mixed-precision refinement of the Laplace form in one
// persistent launch.  The queue holds two jobs per block: the solve jobs in
// the dataflow order of a solve, and, `lag` solve jobs behind, the residual
// jobs interleaved with them (S_0 .. S_{lag-1}, S_lag, R_0, S_lag+1, R_1, ...):
//   solve job:    the FP32 solve of the block (the same per-block function as
//                 a solve), X += s D on the block (FP64) with its float-pair
//                 split, then publication of the block (its "solved" flag);
//   residual job: the double-float residual R = B - A(X) of the block.  It
//                 reads the blocks on the block's mode lines with a larger or
//                 equal index -- the block itself and its solve's sources, all
//                 solved before it -- so it waits for the block's own flag only.
// By the time R_i is taken, block i has normally been solved, so residual
// jobs (bound by the FP32 pipes) fill the SM time the latency-bound solve
// leaves idle instead of queueing after it.
#pragma once

#include "apply_tile.cuh"
#include "batched.h"
#include "fused.h"
#include "wave_kernel.cuh"

namespace tsylv {

template <int D>
struct FusedCfg {
    using CW = WaveCfg<float, D, false>;
    using CA = apply_detail::ApplyCfg<D, apply_detail::kModeDF>;
    static constexpr size_t body = CW::smem > CA::smem ? CW::smem : CA::smem;
    static constexpr size_t oBarW = (body + 15) / 16 * 16;
    static constexpr size_t oBarA = oBarW + 8 * CW::NST;
    static constexpr size_t smem = oBarA + 8 * CA::NST;
};

template <int D>
__global__ void __launch_bounds__(kThreads) k_fused_step(const FusedArgs f) {
    using F = FusedCfg<D>;
    using CW = typename F::CW;
    using CA = typename F::CA;
    constexpr int TD = CW::TD;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* barW = reinterpret_cast<uint64_t*>(smem_raw + F::oBarW);
    uint64_t* barA = reinterpret_cast<uint64_t*>(smem_raw + F::oBarA);
    __shared__ int s_job;
    __shared__ double s_red[kThreads / 32];
    if (threadIdx.x == 0) {
        for (int q = 0; q < CW::NST; q++) dev::mbar_init(&barW[q], 1);
        for (int q = 0; q < CA::NST; q++) dev::mbar_init(&barA[q], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t usesW[CW::NST] = {};
    uint32_t usesA[CA::NST] = {};
    bool alive = true;
    const WaveArgs& a = f.b.eqs[0];
    const double sc = dev::step_scale(f.nrm[1]);
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(f.b.head, 1);
        __syncthreads();
        const int j = s_job;
        const int N = f.b.njobs, K = f.lag < N ? f.lag : N;
        if (j >= 2 * N) break;
        // job j -> solve job or residual job of the queue position's block
        int idx;
        bool resid;
        if (j < K) {
            idx = j;
            resid = false;
        } else if (j < K + 2 * (N - K)) {
            const int r = j - K;
            resid = r & 1;
            idx = resid ? r >> 1 : K + (r >> 1);
        } else {
            idx = (N - K) + (j - K - 2 * (N - K));
            resid = true;
        }
        if (resid) {
            const long long t = f.b.tiles[idx];
            if (threadIdx.x == 0) {
                if (!dev::wait_at_least(a.ready + t, 1, f.b.abort, f.b.timeout_ns)) atomicOr(a.err, kErrTimeout);
                dev::fence_proxy_async_all();
            }
            __syncthreads();
            if (alive) apply_detail::apply_tile<D, apply_detail::kModeDF>(f.ap, t, smem_raw, barA, usesA);
            __syncthreads();
            continue;
        }
        const long long t = f.b.tiles[idx];
        if (alive) alive = wave_tile<float, D, false>(a, t, 0, 1, usesW, barW);
        __syncthreads();
        // X += s D on the block, its split, and the block's sum of X^2
        const float* Dt = static_cast<const float*>(a.X) + t * TD;
        double ss = 0;
        for (int e = threadIdx.x; e < TD; e += kThreads) {
            const long long i = t * TD + e;
            const double v = f.X[i] + sc * static_cast<double>(Dt[e]);
            f.X[i] = v;
            const float hv = static_cast<float>(v);
            f.Xh[i] = hv;
            f.Xl[i] = static_cast<float>(v - static_cast<double>(hv));
            ss += v * v;
        }
        for (int w = 16; w >= 1; w >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, w);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ss;
        // publish the block (every thread's stores, then the flag); the
        // residual below reads the split through bulk copies (async proxy)
        __threadfence();
        dev::fence_proxy_async_all();
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0;
            for (int w = 0; w < kThreads / 32; w++) tot += s_red[w];
            f.xpart[t] = tot;
            dev::st_release(const_cast<int*>(a.ready) + t, 1);
        }
        __syncthreads();
    }
}

template <int D>
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
            if (alive) alive = wave_tile<float, D, false>(kind == 0 ? w1 : w2, t, 0, 1, usesW, barW);
            __syncthreads();
            if (threadIdx.x == 0) dev::publish(const_cast<int*>((kind == 0 ? w1 : w2).ready) + t, 1, nullptr);
        } else if (kind == 1) {
            if (alive) apply_detail::apply_tile<D, apply_detail::kModeDFh>(f.r1, t, smem_raw, barA, usesA);
            __syncthreads();
            // right-hand side of the second solve: R1 / s (exact scaling)
            const double* R = f.r1.R + t * TD;
            for (int e = threadIdx.x; e < TD; e += kThreads) f.X2[t * TD + e] = static_cast<float>(R[e]) * inv;
            __syncthreads();
            if (threadIdx.x == 0) dev::publish(f.r1done + t, 1, nullptr);
        } else {
            if (alive) apply_detail::apply_tile<D, apply_detail::kModeF32>(f.r2, t, smem_raw, barA, usesA);
            __syncthreads();
        }
    }
}

template <int D>
int refine2_occupancy_t() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refine2<D>, kThreads, FusedCfg<D>::smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <int D>
cudaError_t launch_refine2_t(const Refine2Args& f, int grid, cudaStream_t s) {
    k_refine2<D><<<grid, kThreads, FusedCfg<D>::smem, s>>>(f);
    return cudaGetLastError();
}

template <int D>
cudaError_t prepare_fused_t() {
    cudaError_t e = cudaFuncSetAttribute(k_fused_step<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(FusedCfg<D>::smem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_refine2<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(FusedCfg<D>::smem));
}

template <int D>
int fused_occupancy_t() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused_step<D>, kThreads, FusedCfg<D>::smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <int D>
cudaError_t launch_fused_t(const FusedArgs& f, int grid, cudaStream_t s) {
    k_fused_step<D><<<grid, kThreads, FusedCfg<D>::smem, s>>>(f);
    return cudaGetLastError();
}

}  // namespace tsylv
