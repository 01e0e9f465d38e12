// Persistent batched solve: CTAs take jobs (one block of one equation each)
// from a global queue in queue order, wait until the block's prerequisite
// wavefronts of its equation are finished, and run the same per-block update
// and base case as a wavefront launch.  Every wait is bounded.
#pragma once

#include "batched.h"
#include "wave_kernel.cuh"

namespace tsylv {

template <typename T, int D, int GENF, int PK = kProdNative>
__global__ void __launch_bounds__(kThreads, WaveCfg<T, D, GENF>::MINB) k_batched(const BatchArgs b) {
    using C = WaveCfg<T, D, GENF>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::oBar);
    __shared__ int s_job, s_ok;
    if (threadIdx.x == 0) {
        for (int q = 0; q < C::NST; q++) dev::mbar_init(&bar[q], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses[C::NST] = {};
    bool alive = true;  // false after a timed-out copy: no further copies on these barriers
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(b.head, 1);
        __syncthreads();
        const int j = s_job;
        if (j >= b.njobs) break;
        BatchJob jb;
        if (b.jobs) {
            jb = b.jobs[j];
        } else {
            jb.eq = 0;
            jb.tile = b.tiles[j];
            jb.need = 0;
        }
        const WaveArgs& a = b.eqs[jb.eq];
        if (threadIdx.x == 0) {
            int ok = 1;
            if (jb.need > 0 && !dev::wait_at_least(&b.done[jb.eq], jb.need, b.abort, b.timeout_ns)) ok = 0;
            if (!ok) atomicOr(a.err, kErrTimeout);
            dev::fence_proxy_async_all();
            s_ok = ok;
        }
        __syncthreads();
        if (alive && s_ok) alive = wave_tile<T, D, GENF, PK>(a, jb.tile, 0, 1, uses, bar);
        // publish the block: every thread's stores, then the count / flag
        // (one release by one thread after the barrier)
        __syncthreads();
        if (threadIdx.x == 0)
            dev::publish(a.ready ? const_cast<int*>(a.ready) + jb.tile : nullptr, 1, b.done ? &b.done[jb.eq] : nullptr);
    }
}

template <typename T, int D, int GEN, int PK = kProdNative>
cudaError_t prepare_batched_t() {
    using C = WaveCfg<T, D, GEN>;
    return cudaFuncSetAttribute(k_batched<T, D, GEN, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::smem));
}

template <typename T, int D, int GEN, int PK = kProdNative>
cudaError_t launch_batched_t(const BatchArgs& a, int grid, cudaStream_t s) {
    using C = WaveCfg<T, D, GEN>;
    k_batched<T, D, GEN, PK><<<grid, kThreads, C::smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int GEN, int PK = kProdNative>
int batched_occupancy_t() {
    using C = WaveCfg<T, D, GEN>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<T, D, GEN, PK>, kThreads, C::smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace tsylv
