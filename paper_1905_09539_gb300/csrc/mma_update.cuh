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
// (m16n8k8, k zero-padded when TE = 4), accumulating in FP32 registers; the
// FP64 solve's variant issues FP64 DMMA (m8n8k4, 8 x 8 output tiles) on FP64
// operands and accumulators, skipping the output tiles whose rows are all
// padding of the target block and the k steps beyond the source block.
// Every accumulator slot of the block update (one per mode for the Laplace
// form, one per Horner level sum for the d-term form) has a fixed mode, hence
// a fixed fragment layout, for the whole block; after the last job the
// fragments are summed into shared memory in element order and handed to the
// base case exactly as the FP32 path hands over its registers.
#pragma once

#include "device_common.cuh"
#include "tsylv_internal.h"

namespace tsylv {

template <bool B, typename X, typename Y>
struct Pick { using type = X; };
template <typename X, typename Y>
struct Pick<false, X, Y> { using type = Y; };

template <int D, int PK>
struct MmaCfg {
    static constexpr bool F64 = PK == kProdDMMA;
    using F = typename Pick<F64, double, float>::type;  // operands and accumulators in shared memory
    static constexpr int TE = tile_extent(D);
    static constexpr int R = ipow(TE, D - 1);            // rows of C: the other modes' indices
    static constexpr int MR = F64 ? 8 : 16;              // rows of an output tile
    static constexpr int NF = F64 ? 2 : 4;               // accumulator entries per thread and tile
    static constexpr int MT = (R + MR - 1) / MR;         // row tiles
    static constexpr int NT = (TE + 7) / 8;              // 8-column tiles
    static constexpr int KSTEP = F64 ? 4 : (PK == kProdTF32 && TE % 8 != 0) ? 4 : 8;
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

// D (8 x 8) += A (8 x 4) B (4 x 8) in FP64: a0 = A(g, t), b0 = B(t, g),
// c = C(g, 2t), C(g, 2t + 1)  (g = lane / 4, t = lane % 4)
__device__ __forceinline__ void mma_f64_k4(double (&c)[2], double a0, double b0) {
    asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(c[0]), "+d"(c[1])
        : "d"(a0), "d"(b0));
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
template <int D, int MU, typename F>
__device__ __forceinline__ F a_at(const F* S, int r, int k) {
    constexpr int TE = tile_extent(D);
    constexpr int R = ipow(TE, D - 1);
    return (r < R && k < TE) ? S[elem_of<D, MU>(r, k)] : F(0);
}

// B(k, n) = M(n, k)
template <int D, typename F>
__device__ __forceinline__ F b_at(const F* M, int k, int n) {
    constexpr int TE = tile_extent(D);
    return (k < TE && n < TE) ? M[n + TE * k] : F(0);
}

}  // namespace mma_detail

// Bit MU * UPW + u: the warp's output tile u of a mode-MU product holds a
// row of the target block (not padding only).  The rows of a tile share
// their slower coordinates and run over consecutive values of the fastest
// one, so the tile is live exactly when its first row is.
template <int D, int PK, int MU = 0>
__device__ __forceinline__ unsigned mma_tile_live(const int* bs) {
    using Q = MmaCfg<D, PK>;
    constexpr int TE = tile_extent(D);
    unsigned bits = 0;
    if constexpr (MU < D) {
        const int warp = threadIdx.x >> 5;
#pragma unroll
        for (int u = 0; u < Q::UPW; u++) {
            const int unit = warp + Q::NW * u;
            if (unit >= Q::UNITS) continue;
            const int ot = unit % Q::OT;
            int e = mma_detail::elem_of<D, MU>((ot / Q::NT) * Q::MR, 0);
            bool live = true;
#pragma unroll
            for (int nu = 0; nu < D; nu++) {
                if (e % TE >= bs[nu]) live = false;
                e /= TE;
            }
            if (live) bits |= 1u << (MU * Q::UPW + u);
        }
        bits |= mma_tile_live<D, PK, MU + 1>(bs);
    }
    return bits;
}

// c[u] += (S x_MU M) on the warp's output units u.  The FP64 variant skips
// the k steps at and beyond the source block's extent ks and the output
// tiles that hold padding only (bits `tl`, mma_tile_live); the TF32 / BF16
// variants compute full tiles.
template <int D, int PK, int MU>
__device__ __forceinline__ void mma_prod(typename MmaCfg<D, PK>::F (&c)[MmaCfg<D, PK>::UPW][MmaCfg<D, PK>::NF],
                                         const typename MmaCfg<D, PK>::F* __restrict__ M,
                                         const typename MmaCfg<D, PK>::F* __restrict__ S, int ks, unsigned tl) {
    using Q = MmaCfg<D, PK>;
    using namespace mma_detail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int u = 0; u < Q::UPW; u++) {
        const int unit = warp + Q::NW * u;
        if (Q::UNITS % Q::NW != 0 && unit >= Q::UNITS) continue;
        const int ot = unit % Q::OT, kp = unit / Q::OT;
        if constexpr (Q::F64) {
            if (!((tl >> (MU * Q::UPW + u)) & 1u)) continue;  // uniform over the warp
            const int r = (ot / Q::NT) * 8 + g;
            const int n = (ot % Q::NT) * 8 + g;
#pragma unroll
            for (int kq = 0; kq < Q::KPER; kq++) {
                const int kb = (kp * Q::KPER + kq) * 4;
                if (kb >= ks) break;
                mma_f64_k4(c[u], a_at<D, MU>(S, r, kb + t), b_at<D>(M, kb + t, n));
            }
        } else {
            const int r0 = (ot / Q::NT) * 16 + g, r1 = r0 + 8;
            const int n = (ot % Q::NT) * 8 + g;
#pragma unroll
            for (int kq = 0; kq < Q::KPER; kq++) {
                const int kb = (kp * Q::KPER + kq) * Q::KSTEP;
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
}

// One block-update job of level L on the tensor cores, the same term pattern
// as the FMA path (JobCompute): Laplace level L is mode L into slot L; the
// d-term form's level L is mode d-1-L into the level's P and G slots.
template <int D, bool GEN, int PK, int L>
struct MmaJob {
    using Q = MmaCfg<D, PK>;
    using F = typename Q::F;
    template <int NS>
    __device__ __forceinline__ static void run(F (&c)[NS][Q::UPW][Q::NF], const F* stage, int ks, unsigned tl) {
        constexpr int TE = tile_extent(D);
        constexpr int TD = ipow(TE, D);
        constexpr int TC = TE * TE;
        const F* S1 = stage;
        const F* S2 = stage + TD;
        const F* M1 = stage + 2 * TD;
        const F* M2 = stage + 2 * TD + TC;
        if constexpr (!GEN) {
            mma_prod<D, PK, L>(c[L], M1, S1, ks, tl);
        } else {
            constexpr int MU = D - 1 - L;
            if constexpr (L == 0) {
                mma_prod<D, PK, MU>(c[0], M1, S1, ks, tl);
                mma_prod<D, PK, MU>(c[1], M2, S1, ks, tl);
            } else if constexpr (MU >= 1) {
                mma_prod<D, PK, MU>(c[2 * L], M1, S1, ks, tl);
                mma_prod<D, PK, MU>(c[2 * L + 1], M1, S2, ks, tl);
                mma_prod<D, PK, MU>(c[2 * L + 1], M2, S1, ks, tl);
            } else {
                mma_prod<D, PK, 0>(c[NS - 1], M1, S2, ks, tl);
                mma_prod<D, PK, 0>(c[NS - 1], M2, S1, ks, tl);
            }
        }
    }
};

template <int D, bool GEN, int PK, int NS, int L = 0>
__device__ __forceinline__ void mma_dispatch(int level,
                                             typename MmaCfg<D, PK>::F (&c)[NS][MmaCfg<D, PK>::UPW][MmaCfg<D, PK>::NF],
                                             const typename MmaCfg<D, PK>::F* stage, int ks, unsigned tl) {
    if constexpr (L < D) {
        if (level == L)
            MmaJob<D, GEN, PK, L>::run(c, stage, ks, tl);
        else
            mma_dispatch<D, GEN, PK, NS, L + 1>(level, c, stage, ks, tl);
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
__device__ __forceinline__ void mma_store(typename MmaCfg<D, PK>::F (&c)[NS][MmaCfg<D, PK>::UPW][MmaCfg<D, PK>::NF],
                                          typename MmaCfg<D, PK>::F* red) {
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
                typename Q::F* dst = red + (GEN ? s * TD : 0);
                const bool first = kp == 0 && (GEN || s == 0);
#pragma unroll
                for (int u = 0; u < Q::UPW; u++) {
                    const int unit = warp + Q::NW * u;
                    if (Q::UNITS % Q::NW != 0 && unit >= Q::UNITS) continue;
                    if (unit / Q::OT != kp) continue;
                    const int ot = unit % Q::OT;
                    const int r0 = (ot / Q::NT) * Q::MR + g;
                    const int n0 = (ot % Q::NT) * 8 + 2 * t;
#pragma unroll
                    for (int h = 0; h < Q::NF; h++) {
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
