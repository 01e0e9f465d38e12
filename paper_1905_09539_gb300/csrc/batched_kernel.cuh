// Persistent batched solve: CTAs take jobs (one block of one equation each)
// from a global queue in queue order, wait until the block's prerequisite
// wavefronts of its equation are finished, and run the same per-block update
// and base case as a wavefront launch.  Every wait is bounded.
#pragma once

#include "batched.h"
#include "wave_kernel.cuh"

namespace tsylv {

namespace dev {

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Order earlier generic-proxy accesses (including what an acquire made
// visible) before later bulk copies, in every state space.
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Wait (bounded) until *p >= need.  A timeout raises *abort, which makes
// every later wait of the launch give up at once.
__device__ __forceinline__ bool wait_count(const int* p, int need, int* abort, long long timeout_ns) {
    if (ld_acquire(p) >= need) return true;
    const unsigned long long t0 = global_ns();
    while (ld_acquire(p) < need) {
        if (ld_acquire(abort) || static_cast<long long>(global_ns() - t0) > timeout_ns) {
            atomicExch(abort, 1);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

}  // namespace dev

template <typename T, int D, bool GENF>
__global__ void __launch_bounds__(kThreads) k_batched(const BatchArgs b) {
    using C = WaveCfg<T, D, GENF>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::oBar);
    __shared__ int s_job, s_ok;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses[2] = {0u, 0u};
    bool alive = true;  // false after a timed-out copy: no further copies on these barriers
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(b.head, 1);
        __syncthreads();
        const int j = s_job;
        if (j >= b.njobs) break;
        const BatchJob jb = b.jobs[j];
        if (threadIdx.x == 0) {
            int ok = 1;
            if (jb.need > 0 && !dev::wait_count(&b.done[jb.eq], jb.need, b.abort, b.timeout_ns)) ok = 0;
            if (!ok) atomicOr(b.eqs[jb.eq].err, kErrTimeout);
            dev::fence_proxy_async_all();
            s_ok = ok;
        }
        __syncthreads();
        if (alive && s_ok) {
            const WaveArgs& a = b.eqs[jb.eq];
            alive = wave_tile<T, D, GENF>(a, jb.tile, 0, 1, uses);
        }
        // publish the block: every thread's stores, then the count (release)
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&b.done[jb.eq], 1);
    }
}

template <typename T, int D, bool GEN>
cudaError_t prepare_batched_t() {
    using C = WaveCfg<T, D, GEN>;
    return cudaFuncSetAttribute(k_batched<T, D, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::smem));
}

template <typename T, int D, bool GEN>
cudaError_t launch_batched_t(const BatchArgs& a, int grid, cudaStream_t s) {
    using C = WaveCfg<T, D, GEN>;
    k_batched<T, D, GEN><<<grid, kThreads, C::smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, bool GEN>
int batched_occupancy_t() {
    using C = WaveCfg<T, D, GEN>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<T, D, GEN>, kThreads, C::smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace tsylv
