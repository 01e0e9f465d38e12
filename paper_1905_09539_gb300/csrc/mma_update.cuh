// Block updates of the low-precision solves on the tensor cores.
//
// The update of Eq. (2.3a) restricted to one block is a sum of block mode
// products  Y += S x_mu M  (M a TE x TE coefficient tile, S a solved source
// block or a Horner intermediate of the d-term form).  Written as a matrix
// product over the other modes' indices r (R = TE^(d-1) rows) it is
//     Y^(r, i) += sum_k S^(r, k) M(i, k),
// i.e. C (R x TE) += A (R x TE) * B (TE x TE) with A = S^ (rows: the other
// modes, columns: the mode-mu index) and B = M^T.  Each warp of the CTA owns
// fixed 16 x 8 output tiles of C (and, when there are fewer tiles than warps,
// a share of the k range) and issues warp-level mma.sync instructions on
// operands rounded to TF32 (m16n8k8, or m16n8k4 when TE = 4) or BF16
// (m16n8k8, k zero-padded when TE = 4), accumulating in FP32 registers.
// Every accumulator slot of the block update (one per mode for the Laplace
// form, one per Horner level sum for the d-term form) has a fixed mode, hence
// a fixed fragment layout, for the whole block; after the last job the
// fragments are summed into shared memory in element order and handed to the
// base case exactly as the FP32 path hands over its registers.
#pragma once

#include "device_common.cuh"
#include "tsylv_internal.h"

namespace tsylv {

template <int D, int PK>
struct MmaCfg {
    static constexpr int TE = tile_extent(D);
    static constexpr int R = ipow(TE, D - 1);            // rows of C: the other modes' indices
    static constexpr int MT = (R + 15) / 16;             // 16-row tiles
    static constexpr int NT = (TE + 7) / 8;              // 8-column tiles
    static constexpr int KSTEP = (PK == kProdTF32 && TE % 8 != 0) ? 4 : 8;
    static constexpr int KS = (TE + KSTEP - 1) / KSTEP;  // k steps over the mode extent
    static constexpr int NW = kThreads / 32;
    static constexpr int OT = MT * NT;
    // when the output tiles alone leave warps idle, the k steps are split too
    static constexpr int KSPLIT = (OT < NW && KS >= NW / OT && KS % (NW / OT) == 0) ? NW / OT : 1;
    static constexpr int KPER = KS / KSPLIT;
    static constexpr int UNITS = OT * KSPLIT;
    static constexpr int UPW = (UNITS + NW - 1) / NW;    // units per warp
    // accumulator slots: Laplace one per mode; d-term one per Horner level sum
    static constexpr int NS_LAP = D;
};

namespace mma_detail {

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// two floats to a bf16 pair: `lo` in the low half (the smaller k index)
__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_tf32_k8(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                            uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32_k4(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm("mma.sync.aligned.m16n8k4.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_bf16_k8(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// In-block element of (row r of the other modes, index i of mode MU).
template <int D, int MU>
__device__ __forceinline__ int elem_of(int r, int i) {
    constexpr int TE = tile_extent(D);
    constexpr int st = ipow(TE, MU);
    return (r % st) + i * st + (r / st) * (st * TE);
}

// S^ (row r, column k), zero outside the block's extent of the matrix
template <int D, int MU>
__device__ __forceinline__ float a_at(const float* S, int r, int k) {
    constexpr int TE = tile_extent(D);
    constexpr int R = ipow(TE, D - 1);
    return (r < R && k < TE) ? S[elem_of<D, MU>(r, k)] : 0.f;
}

// B(k, n) = M(n, k)
template <int D>
__device__ __forceinline__ float b_at(const float* M, int k, int n) {
    constexpr int TE = tile_extent(D);
    return (k < TE && n < TE) ? M[n + TE * k] : 0.f;
}

}  // namespace mma_detail

// c[u] += (S x_MU M) on the warp's output units u.
template <int D, int PK, int MU>
__device__ __forceinline__ void mma_prod(float (&c)[MmaCfg<D, PK>::UPW][4], const float* __restrict__ M,
                                         const float* __restrict__ S) {
    using Q = MmaCfg<D, PK>;
    using namespace mma_detail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int u = 0; u < Q::UPW; u++) {
        const int unit = warp + Q::NW * u;
        if (Q::UNITS % Q::NW != 0 && unit >= Q::UNITS) continue;
        const int ot = unit % Q::OT, kp = unit / Q::OT;
        const int r0 = (ot / Q::NT) * 16 + g, r1 = r0 + 8;
        const int n = (ot % Q::NT) * 8 + g;
#pragma unroll
        for (int ks = 0; ks < Q::KPER; ks++) {
            const int kb = (kp * Q::KPER + ks) * Q::KSTEP;
            if constexpr (PK == kProdTF32 && Q::KSTEP == 8) {
                mma_tf32_k8(c[u], to_tf32(a_at<D, MU>(S, r0, kb + t)), to_tf32(a_at<D, MU>(S, r1, kb + t)),
                            to_tf32(a_at<D, MU>(S, r0, kb + t + 4)), to_tf32(a_at<D, MU>(S, r1, kb + t + 4)),
                            to_tf32(b_at<D>(M, kb + t, n)), to_tf32(b_at<D>(M, kb + t + 4, n)));
            } else if constexpr (PK == kProdTF32) {
                mma_tf32_k4(c[u], to_tf32(a_at<D, MU>(S, r0, kb + t)), to_tf32(a_at<D, MU>(S, r1, kb + t)),
                            to_tf32(b_at<D>(M, kb + t, n)));
            } else {
                const int k0 = kb + 2 * t;
                mma_bf16_k8(c[u], to_bf16x2(a_at<D, MU>(S, r0, k0), a_at<D, MU>(S, r0, k0 + 1)),
                            to_bf16x2(a_at<D, MU>(S, r1, k0), a_at<D, MU>(S, r1, k0 + 1)),
                            to_bf16x2(b_at<D>(M, k0, n), b_at<D>(M, k0 + 1, n)));
            }
        }
    }
}

// One block-update job of level L on the tensor cores, the same term pattern
// as the FP32 path (JobCompute): Laplace level L is mode L into slot L; the
// d-term form's level L is mode d-1-L into the level's P and G slots.
template <int D, bool GEN, int PK, int L>
struct MmaJob {
    template <int NS>
    __device__ __forceinline__ static void run(float (&c)[NS][MmaCfg<D, PK>::UPW][4], const float* stage) {
        constexpr int TE = tile_extent(D);
        constexpr int TD = ipow(TE, D);
        constexpr int TC = TE * TE;
        const float* S1 = stage;
        const float* S2 = stage + TD;
        const float* M1 = stage + 2 * TD;
        const float* M2 = stage + 2 * TD + TC;
        if constexpr (!GEN) {
            mma_prod<D, PK, L>(c[L], M1, S1);
        } else {
            constexpr int MU = D - 1 - L;
            if constexpr (L == 0) {
                mma_prod<D, PK, MU>(c[0], M1, S1);
                mma_prod<D, PK, MU>(c[1], M2, S1);
            } else if constexpr (MU >= 1) {
                mma_prod<D, PK, MU>(c[2 * L], M1, S1);
                mma_prod<D, PK, MU>(c[2 * L + 1], M1, S2);
                mma_prod<D, PK, MU>(c[2 * L + 1], M2, S1);
            } else {
                mma_prod<D, PK, 0>(c[NS - 1], M1, S2);
                mma_prod<D, PK, 0>(c[NS - 1], M2, S1);
            }
        }
    }
};

template <int D, bool GEN, int PK, int NS, int L = 0>
__device__ __forceinline__ void mma_dispatch(int level, float (&c)[NS][MmaCfg<D, PK>::UPW][4], const float* stage) {
    if constexpr (L < D) {
        if (level == L)
            MmaJob<D, GEN, PK, L>::run(c, stage);
        else
            mma_dispatch<D, GEN, PK, NS, L + 1>(level, c, stage);
    }
}

// Mode of accumulator slot s.
template <int D, bool GEN>
__host__ __device__ constexpr int mma_slot_mode(int s) {
    return GEN ? D - 1 - (s >> 1) : s;
}

// Sum the fragments into red (element order): the d-term form's slots into
// red[s * TD + e], the Laplace form's per-mode slots all into red[e].  Units
// of different k parts, and the Laplace slots, are added one pass after the
// other (a CTA barrier between passes), so every entry has one writer per pass.
template <int D, bool GEN, int PK, int NS>
__device__ __forceinline__ void mma_store(float (&c)[NS][MmaCfg<D, PK>::UPW][4], float* red) {
    using Q = MmaCfg<D, PK>;
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    constexpr int SP = GEN ? 1 : NS;  // slot passes
#pragma unroll
    for (int sp = 0; sp < SP; sp++)
#pragma unroll
        for (int kp = 0; kp < Q::KSPLIT; kp++) {
            __syncthreads();
#pragma unroll
            for (int s = 0; s < NS; s++) {
                if (!GEN && s != sp) continue;
                float* dst = red + (GEN ? s * TD : 0);
                const bool first = kp == 0 && (GEN || s == 0);
#pragma unroll
                for (int u = 0; u < Q::UPW; u++) {
                    const int unit = warp + Q::NW * u;
                    if (Q::UNITS % Q::NW != 0 && unit >= Q::UNITS) continue;
                    if (unit / Q::OT != kp) continue;
                    const int ot = unit % Q::OT;
                    const int r0 = (ot / Q::NT) * 16 + g;
                    const int n0 = (ot % Q::NT) * 8 + 2 * t;
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const int r = r0 + (h >> 1) * 8, i = n0 + (h & 1);
                        if (r >= Q::R || i >= TE) continue;
                        int e;
                        switch (mma_slot_mode<D, GEN>(s)) {
                            case 0: e = mma_detail::elem_of<D, 0>(r, i); break;
                            case 1: e = mma_detail::elem_of<D, (D > 1 ? 1 : 0)>(r, i); break;
                            case 2: e = mma_detail::elem_of<D, (D > 2 ? 2 : 0)>(r, i); break;
                            case 3: e = mma_detail::elem_of<D, (D > 3 ? 3 : 0)>(r, i); break;
                            default: e = mma_detail::elem_of<D, (D > 4 ? 4 : 0)>(r, i); break;
                        }
                        dst[e] = first ? c[s][u][h] : dst[e] + c[s][u][h];
                    }
                }
            }
        }
    __syncthreads();
}

}  // namespace tsylv
