// PTX helpers for sm_103a: bulk (TMA) copies with mbarrier completion,
// thread-block clusters and distributed shared memory.  Every wait is
// bounded by a %globaltimer deadline.
#pragma once

#include <cstdint>

#include "complex_z.h"
#include "double_float.h"

namespace tsylv {
namespace dev {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async proxy and the cluster.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this CTA's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes into the same buffer.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bulk global -> shared copy (the untiled TMA path).  dst, src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `parity` to complete; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (static_cast<long long>(global_ns() - t0) > timeout_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_rank(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(local)), "r"(rank));
    return r;
}

__device__ __forceinline__ double ld_dsmem(const double* local, uint32_t rank) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(map_rank(local, rank)) : "memory");
    return v;
}
__device__ __forceinline__ float ld_dsmem(const float* local, uint32_t rank) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(map_rank(local, rank)) : "memory");
    return v;
}

// ---- inter-CTA signalling through global memory (persistent kernels)

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_relaxed_add(int* p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Acquire-release fence at GPU scope: after a relaxed load that saw a flag
// it completes an acquire; before relaxed stores it makes them a release
// (cumulative: it covers what the CTA's barrier ordered before it).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Publish a CTA's results: after a barrier of the CTA, one thread makes every
// thread's earlier stores visible at GPU scope before the flag (and counter).
__device__ __forceinline__ void publish(int* flag, int v, int* counter) {
    fence_acq_rel_gpu();
    if (counter) red_relaxed_add(counter, 1);
    if (flag) st_relaxed(flag, v);
}

// Order earlier generic-proxy accesses (including what an acquire made
// visible) before later bulk copies, in every state space.
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Wait (bounded) until *p >= need: relaxed polls (one L2 round trip each,
// no sleep), then an acquire fence.  A timeout raises *abort, which makes
// every later wait of the launch give up at once.  Returns false on either.
__device__ __forceinline__ bool wait_at_least(const int* p, int need, int* abort, long long timeout_ns) {
    if (ld_acquire(p) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; it++) {
        if (ld_relaxed(p) >= need) break;
        if ((it & 15u) == 0 &&
            (ld_relaxed(abort) || static_cast<long long>(global_ns() - t0) > timeout_ns)) {
            atomicExch(abort, 1);
            return false;
        }
    }
    fence_acq_rel_gpu();
    return true;
}

// Scale of a refinement step: the power of two at or above max|R| (1 when R
// is zero or not finite), so that R / s and s * D are exact.
__device__ __forceinline__ double step_scale(double mx) {
    if (!(mx > 0) || !::isfinite(mx)) return 1.0;
    int ex = 0;
    (void)frexp(mx, &ex);  // mx = f 2^ex, 1/2 <= f < 1
    return ldexp(1.0, ex);
}

// a + b rounded on its own (the compiler may not fuse it with the product
// that produced a or b)
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T fmadd(T a, T b, T c);
template <>
__device__ __forceinline__ double fmadd<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct Eps;
template <>
struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <>
struct Eps<float> { static constexpr float v = 1.1920929e-07f; };
template <>
struct Eps<zd> { static constexpr double v = 2.220446049250313e-16; };

// complex multiply-add c + a b as four real fused multiply-adds
template <>
__device__ __forceinline__ zd fmadd<zd>(zd a, zd b, zd c) {
    return zd(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}
__device__ __forceinline__ zd add_rn(zd a, zd b) { return zd(__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im)); }
__device__ __forceinline__ zd ld_dsmem(const zd* local, uint32_t rank) {
    return zd(ld_dsmem(&local->re, rank), ld_dsmem(&local->im, rank));
}

// Double-float: epsilon of the pair arithmetic (2^-44, a bound on the
// relative error of one operation); the block products accumulate with a
// multiply-add that leaves its pair unnormalised (the high words summed by
// two_sum, every error and low-word product gathered in the low word), and
// `settle` normalises an accumulator once its products are summed.
template <>
struct Eps<dfl> { static constexpr float v = 5.684341886080802e-14f; };
template <>
__device__ __forceinline__ dfl fmadd<dfl>(dfl a, dfl b, dfl c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);  // exact: a.h b.h = p + e
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    float s, t;
    dfl_detail::two_sum(c.h, p, s, t);
    return dfl(s, __fadd_rn(t, __fadd_rn(c.l, e)));
}
__device__ __forceinline__ dfl add_rn(dfl a, dfl b) { return a + b; }
__device__ __forceinline__ dfl ld_dsmem(const dfl* local, uint32_t rank) {
    return dfl(ld_dsmem(&local->h, rank), ld_dsmem(&local->l, rank));
}
template <typename T>
__device__ __forceinline__ T settle(T x) { return x; }

// warp broadcast of a value of the element type (within segments of `width`
// lanes when width < 32: src is then the lane within the segment)
template <typename T>
__device__ __forceinline__ T shfl(unsigned mask, T v, int src, int width = 32) {
    return __shfl_sync(mask, v, src, width);
}
template <>
__device__ __forceinline__ dfl shfl<dfl>(unsigned mask, dfl v, int src, int width) {
    return dfl(__shfl_sync(mask, v.h, src, width), __shfl_sync(mask, v.l, src, width));
}
template <>
__device__ __forceinline__ zd shfl<zd>(unsigned mask, zd v, int src, int width) {
    return zd(__shfl_sync(mask, v.re, src, width), __shfl_sync(mask, v.im, src, width));
}
template <>
__device__ __forceinline__ dfl settle<dfl>(dfl x) { return dfl_detail::fast_two_sum(x.h, x.l); }

}  // namespace dev
}  // namespace tsylv
