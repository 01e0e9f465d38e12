// Wavefront kernel: for every block T of one anti-diagonal of the block grid,
//   1. the right-hand-side update of Eq. (2.3a) restricted to T: block
//      mode-mu products of already solved blocks with the off-diagonal
//      coefficient blocks A_mu(I, J') (Laplace form), or -- generalized
//      d-term form -- the same updates organised as a Horner recurrence over
//      the modes (intermediates P_l, G_l), the term pattern of Sec. 3.1;
//   2. the base case: the diagonal-block equation of T solved by
//      back-substitution over the coupled groups (products of the 1x1/2x2
//      Schur blocks of every mode), i.e. the merged-mode solve of Alg. 3 in
//      which the diagonal blocks after the perfect shuffle (Sec. 2.3) are
//      solved directly.
// Step 1 is split over a thread-block cluster of `csize` CTAs (disjoint
// source ranges, bulk-copied through shared memory); the partial sums are
// reduced through distributed shared memory into rank 0, which performs
// step 2.
#pragma once

#include "device_common.cuh"
#include "mma_update.cuh"
#include "tsylv_internal.h"

namespace tsylv {

// Forms (kForm*, tsylv_internal.h): the two-term form Eq. (3.1) is
// X x_1 A_1 + X x_1 C x_2 A_2 ... x_d A_d.
template <typename T, int D, int FM>
struct WaveCfg {
    static constexpr int TE = tile_extent(D);
    static constexpr int TD = ipow(TE, D);
    static constexpr int TC = TE * TE;
    static constexpr int EPT = (TD + kThreads - 1) / kThreads;
    static constexpr bool GEN = FM == kFormDTerm && D >= 2;
    static constexpr bool TT = FM == kFormTwoTerm && D >= 2;
    static constexpr bool CHAIN = GEN || TT;  // Horner chain over the modes, stored intermediates
    // accumulator slots: Laplace one; d-term P_l, G_l (l = d-1..1) and the
    // mode-1 level; two-term Q_l (l = d-1..1, slot d-1-l) and the mode-1 level
    static constexpr int NACC = GEN ? 2 * (D - 1) + 1 : TT ? D : 1;
    static constexpr int NL = CHAIN ? D - 1 : 0;  // stored levels l = 1..d-1
    static constexpr int STAGE = 2 * TD + 2 * TC;
    // stages of the bulk-copy ring: the FP64 updates are bound by the FP64
    // pipes; the FP32 solves of d = 3 measured faster with 2 stages and more
    // resident CTAs than with 4 (other orders keep 4)
    static constexpr int NST = (sizeof(T) >= 8 || D == 3) ? 2 : 4;
    // resident CTAs per SM the persistent kernel is compiled for (register
    // budget): FP64 Laplace d = 3 6 (its shared memory allows 6, registers
    // alone would give 5), FP64 generalized 3 (shared-memory bound); FP32
    // d = 3 8 (Laplace) / 5 (generalized), other orders 5 / 4
    static constexpr int MINB = D == 5 ? 3  // d = 5: 1024-entry blocks, shared memory allows 3 CTAs/SM
                                : sizeof(T) == 16 ? 3  // complex FP64: 16-byte entries
                                // double-float: the Laplace form measured fastest at 5 (10.6 ms at
                                // 256^3 against 11.5 at 4 and 10.8 at 6); the d-term form is
                                // shared-memory bound at 3
                                : IsDoubleFloat<T>::value ? (CHAIN ? 3 : 5)
                                : sizeof(T) == 8 ? (CHAIN ? (D == 3 ? 3 : 4) : (D == 3 ? 6 : 4))
                                : D == 3 ? (CHAIN ? 5 : 8)
                                         : (CHAIN ? 4 : 5);
    // The coupled-group inverses depend only on the diagonal blocks: they are
    // computed when the block starts, off the critical path, in a region of
    // their own (INV_EARLY), except for the FP64 Laplace form, whose shared
    // memory budget (6 resident CTAs) keeps them in the staging ring (so does d = 1), computed
    // after the block updates.  The FP64 generalized form's in-block
    // intermediates Pin, Gin (base case only) use the staging ring instead.
    // The base case's running line sums of coupled-group members reuse the
    // block-update sums `red` once those are consumed (the generalized form's
    // level sums are parked in the output P, G blocks meanwhile), and the
    // reciprocal diagonal of a 1x1 group sits in its not yet solved X entry.
    static constexpr int MINV = 1024;  // budget (entries) for precomputed coupled-group inverses
    // (complex triangular coefficients have no 2x2 blocks, hence no inverses)
    static constexpr bool CPLX = IsComplex<T>::value;
    static constexpr bool INV_EARLY = D >= 2 && !CPLX && !(sizeof(T) == 8 && !CHAIN);
    // FP64: the base case's line sums run, warp by warp, over the terms some
    // lane of the warp needs (a rolled range; measured 2% faster for the
    // d-term form at 256^3, 2.6% slower for the double-float Laplace form,
    // whose pair arithmetic issues from the FP32 pipes and wants the unrolled,
    // per-lane form)
    static constexpr bool WARP_TERMS = std::is_same<T, double>::value;
    static constexpr bool PIN_IN_RING = CHAIN && sizeof(T) == 8 && 2 * NL * TD <= NST * STAGE;
    static constexpr int UNION = (NST * STAGE > MINV || INV_EARLY) ? NST * STAGE : MINV;
    static constexpr int oStage = 0;
    static constexpr int oRed = UNION;
    static constexpr int oLin = oRed;
    static constexpr int oR = oRed + NACC * TD;
    static constexpr int oX = oR + TD;
    static constexpr int oRd = oX;
    static constexpr int oPin = PIN_IN_RING ? 0 : oX + TD;
    static constexpr int oGin = oPin + NL * TD;
    static constexpr int oD = PIN_IN_RING ? oX + TD : oGin + NL * TD;
    static constexpr int oE = oD + D * TC;
    static constexpr int oMinv = INV_EARLY ? oE + (CHAIN ? D * TC : 0) : 0;
    static constexpr int oEnd = INV_EARLY ? oMinv + MINV : oE + (CHAIN ? D * TC : 0);
    static constexpr size_t oBar = ((oEnd * sizeof(T)) + 15) / 16 * 16;
    static constexpr size_t oMeta = oBar + ((8 * NST + 15) / 16) * 16;
    // meta: gs, gl, gidx [D][TE]; ng, bs [D]; flag [4]; coupled-group lists;
    // element lists
    static constexpr int MAXSTEP = D * TE;
    static constexpr size_t oJob =
        oMeta + (3 * D * TE + 3 * D + 4 + 3 * MAXSTEP + 1 + 2 * (TD / 2 + 1) + 3 * MAXSTEP + 1 + TD) * sizeof(int);
    // decoded jobs (level << 24 | source block) and "source solved" bits of the
    // first JT jobs of a block, filled by all threads at once
    static constexpr int JT = kThreads;
    static constexpr size_t smem = oJob + (JT + JT / 32) * sizeof(int);
    static constexpr int slotP(int l) { return TT ? D - 1 - l : 2 * (D - 1 - l); }
    static constexpr int slotG(int l) { return 2 * (D - 1 - l) + 1; }
};

// acc[q] += (S x_MU M)[e_q] for the thread's elements e_q = tid + q*kThreads:
//   y(.., i, ..) = sum_k M(i, k) S(.., k, ..),  M a TE x TE column-major tile.
// Padding is skipped: k runs over the source block's extent ks in mode MU
// (the tile beyond it is zero), and element slots q whose whole warp holds
// only padded elements of the target block (bit q of `live` clear) are not
// computed (their sums stay zero, as the products of zero padding would be).
// Double-float: one multiply-add is a dozen FP32 instructions, so the k loop
// stays rolled (the fully unrolled products of every level overflow the
// instruction cache) and runs outside the element slots, whose independent
// accumulators then interleave.
template <typename T, int D, int MU, int EPT, int NPROD>
__device__ __forceinline__ void prod_acc_rolled(T (&acc)[EPT], const T* __restrict__ M1, const T* __restrict__ S1,
                                                const T* __restrict__ M2, const T* __restrict__ S2, int ks,
                                                unsigned live) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int st = ipow(TE, MU);
    int iq[EPT], bq[EPT];
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        iq[q] = row_of<TE, st>(e);
        bq[q] = e - iq[q] * st;
    }
#pragma unroll 1  // measured: unrolled by 2 or 4 the solve is 1-55% slower (instruction cache)
    for (int k = 0; k < ks; k++) {
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int e = threadIdx.x + q * kThreads;
            if ((TD % kThreads) != 0 && e >= TD) continue;
            if (!((live >> q) & 1u)) continue;  // uniform over the warp
            acc[q] = dev::fmadd(M1[iq[q] + TE * k], S1[bq[q] + k * st], acc[q]);
            if constexpr (NPROD == 2) acc[q] = dev::fmadd(M2[iq[q] + TE * k], S2[bq[q] + k * st], acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < EPT; q++) acc[q] = dev::settle(acc[q]);
}

template <typename T, int D, int MU, int EPT>
__device__ __forceinline__ void prod_acc(T (&acc)[EPT], const T* __restrict__ M, const T* __restrict__ S, int ks,
                                         unsigned live) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int st = ipow(TE, MU);
    if constexpr (IsDoubleFloat<T>::value) {
        prod_acc_rolled<T, D, MU, EPT, 1>(acc, M, S, M, S, ks, live);
        return;
    }
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        if (!((live >> q) & 1u)) continue;  // uniform over the warp
        const int i = row_of<TE, st>(e);
        const int base = e - i * st;
        T s = acc[q];
        if (ks == TE) {
#pragma unroll
            for (int k = 0; k < TE; k++) s = dev::fmadd(M[i + TE * k], S[base + k * st], s);
        } else {
            for (int k = 0; k < ks; k++) s = dev::fmadd(M[i + TE * k], S[base + k * st], s);
        }
        acc[q] = dev::settle(s);
    }
}

// acc[q] += (S1 x_MU M1 + S2 x_MU M2)[e_q], padding skipped as above
template <typename T, int D, int MU, int EPT>
__device__ __forceinline__ void prod_acc2(T (&acc)[EPT], const T* __restrict__ M1, const T* __restrict__ S1,
                                          const T* __restrict__ M2, const T* __restrict__ S2, int ks,
                                          unsigned live) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int st = ipow(TE, MU);
    if constexpr (IsDoubleFloat<T>::value) {
        prod_acc_rolled<T, D, MU, EPT, 2>(acc, M1, S1, M2, S2, ks, live);
        return;
    }
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        if (!((live >> q) & 1u)) continue;
        const int i = row_of<TE, st>(e);
        const int base = e - i * st;
        T s = acc[q];
        if (ks == TE) {
#pragma unroll
            for (int k = 0; k < TE; k++) {
                s = dev::fmadd(M1[i + TE * k], S1[base + k * st], s);
                s = dev::fmadd(M2[i + TE * k], S2[base + k * st], s);
            }
        } else {
            for (int k = 0; k < ks; k++) {
                s = dev::fmadd(M1[i + TE * k], S1[base + k * st], s);
                s = dev::fmadd(M2[i + TE * k], S2[base + k * st], s);
            }
        }
        acc[q] = dev::settle(s);
    }
}

// Compile-time dispatch of one block-update job of level L.
template <typename T, int D, int FM, int L>
struct JobCompute {
    template <int NACC, int EPT>
    __device__ __forceinline__ static void run(T (&acc)[NACC][EPT], const T* stage, int ks, unsigned live) {
        constexpr int TE = tile_extent(D);
        constexpr int TD = ipow(TE, D);
        constexpr int TC = TE * TE;
        using C = WaveCfg<T, D, FM>;
        const T* S1 = stage;
        const T* S2 = stage + TD;
        const T* M1 = stage + 2 * TD;
        const T* M2 = stage + 2 * TD + TC;
        if constexpr (C::TT) {
            constexpr int MU = D - 1 - L;            // modes d-1, ..., 0
            if constexpr (MU >= 1) {
                // L^Q_mu += Q_{mu+1} x A_mu  (Q_d = X)
                prod_acc<T, D, MU, EPT>(acc[L], M1, S1, ks, live);
            } else {
                // L_0 += Q_1 x C + X x A_1
                prod_acc2<T, D, 0, EPT>(acc[NACC - 1], M1, S2, M2, S1, ks, live);
            }
        } else if constexpr (!C::GEN) {
            prod_acc<T, D, L, EPT>(acc[0], M1, S1, ks, live);  // Laplace: level L = mode L
        } else {
            constexpr int MU = D - 1 - L;            // modes d-1, ..., 0
            if constexpr (L == 0) {
                // L^P_{d-1} += X x C,  L^G_{d-1} += X x A
                prod_acc<T, D, MU, EPT>(acc[0], M1, S1, ks, live);
                prod_acc<T, D, MU, EPT>(acc[1], M2, S1, ks, live);
            } else if constexpr (MU >= 1) {
                // L^P_mu += P_{mu+1} x C,  L^G_mu += G_{mu+1} x C + P_{mu+1} x A
                prod_acc<T, D, MU, EPT>(acc[2 * L], M1, S1, ks, live);
                prod_acc2<T, D, MU, EPT>(acc[2 * L + 1], M1, S2, M2, S1, ks, live);
            } else {
                // L_0 += G_1 x C_0 + P_1 x A_0
                prod_acc2<T, D, 0, EPT>(acc[NACC - 1], M1, S2, M2, S1, ks, live);
            }
        }
    }
};

template <typename T, int D, int FM, int L = 0>
__device__ __forceinline__ void dispatch_job(int level, T (&acc)[WaveCfg<T, D, FM>::NACC][WaveCfg<T, D, FM>::EPT],
                                             const T* stage, int ks, unsigned live) {
    if constexpr (L < D) {
        if (level == L)
            JobCompute<T, D, FM, L>::run(acc, stage, ks, live);
        else
            dispatch_job<T, D, FM, L + 1>(level, acc, stage, ks, live);
    }
}

// Packed per-element data of the back-substitution, built once per block:
// the in-block element (12 bits), whether it belongs to a coupled group, and
// for every mode the first in-block index beyond the element's group (the
// start of its line sums), so that a step reads no group tables.
template <int D>
struct ElemCode {
    static constexpr int TE = tile_extent(D);
    static constexpr int KB = TE >= 32 ? 6 : TE >= 16 ? 5 : TE >= 8 ? 4 : 3;  // bits of a value in [0, TE]
    static_assert(ipow(TE, D) <= 4096 && 13 + KB * D <= 31, "element code does not fit in 31 bits");
    template <typename F>
    __device__ static int make(int e, bool coupled, F k0_of) {
        int c = e | (coupled ? 1 << 12 : 0);
#pragma unroll
        for (int mu = 0; mu < D; mu++) c |= k0_of(mu) << (13 + KB * mu);
        return c;
    }
    __device__ static int elem(int c) { return c & 0xfff; }
    __device__ static bool coupled(int c) { return (c >> 12) & 1; }
    __device__ static int k0(int c, int mu) { return (c >> (13 + KB * mu)) & ((1 << KB) - 1); }
};

template <typename T, int D, int FM>
struct TileSmem {
    const T* Ds;   // [D][TC] diagonal tiles of A
    const T* Es;   // [D][TC] diagonal tiles of C (d-term form) / of the chain factor
                   // (two-term form: C in mode 1, A_mu in the others)
    const T* Rs;   // right-hand side of the diagonal-block equation
    const T* Rd;   // reciprocal of the diagonal entry of every 1x1 group
    T* Xs;         // solution (0 where not yet solved)
    T* Pin;        // [NL][TD] in-block intermediates (generalized)
    T* Gin;
    T* Lin;        // [NACC][TD] running line sums from solved groups
    const int* gs; // [D][TE] group start
    const int* gl; // [D][TE] group length (1 or 2)
    const int* ng; // [D] groups per mode
    const int* bs; // [D] block extent
    const int* gidx; // [D][TE] group of every in-block index
};

// One unknown whose group is 1x1 in every mode: all contributions of solved
// groups are already in the running line sums Lin, so the solve is the
// Horner chain over the diagonal entries (generalized form) and one product
// with the reciprocal diagonal.
template <typename T, int D, int FM>
__device__ __forceinline__ int solve_single(const TileSmem<T, D, FM>& sm, int o, const int (&u)[D],
                                            const T (&L)[WaveCfg<T, D, FM>::NACC]) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int TC = TE * TE;
    using C = WaveCfg<T, D, FM>;
    T x;
    if constexpr (C::TT) {
        // Horner chain of the line sums through the own diagonal entries of the
        // chain factors: Q_l(u) = e_l Q_{l+1}(u) + L_l, Q_d = x; then
        // a_1 x + c Q_1(u) + L_0 = r
        T p0 = L[C::slotP(D - 1)];
        T P0s[D];
        P0s[D - 1] = p0;
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            p0 = dev::fmadd(sm.Es[l * TC + u[l] * (TE + 1)], p0, L[C::slotP(l)]);
            P0s[l] = p0;
        }
        const T off = dev::fmadd(sm.Es[u[0] * (TE + 1)], p0, L[C::NACC - 1]);
        x = (sm.Rs[o] - off) * sm.Rd[o];
        const T e1 = sm.Es[(D - 1) * TC + u[D - 1] * (TE + 1)];
        T pc = e1 * x;
        sm.Pin[(D - 2) * TD + o] = dev::fmadd(e1, x, P0s[D - 1]);
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const T ep = sm.Es[l * TC + u[l] * (TE + 1)];
            sm.Pin[(l - 1) * TD + o] = dev::fmadd(ep, pc, P0s[l]);
            pc = ep * pc;
        }
    } else if constexpr (!C::GEN) {
        x = (sm.Rs[o] - L[0]) * sm.Rd[o];
    } else {
        T p0 = L[C::slotP(D - 1)];
        T g0 = L[C::slotG(D - 1)];
        T P0s[D], G0s[D];
        P0s[D - 1] = p0;
        G0s[D - 1] = g0;
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const T ep = sm.Es[l * TC + u[l] * (TE + 1)], dp = sm.Ds[l * TC + u[l] * (TE + 1)];
            const T np = dev::fmadd(ep, p0, L[C::slotP(l)]);
            const T ng_ = dev::fmadd(ep, g0, dev::fmadd(dp, p0, L[C::slotG(l)]));
            p0 = np;
            g0 = ng_;
            P0s[l] = p0;
            G0s[l] = g0;
        }
        const T off = dev::fmadd(sm.Es[u[0] * (TE + 1)], g0, dev::fmadd(sm.Ds[u[0] * (TE + 1)], p0, L[C::NACC - 1]));
        x = (sm.Rs[o] - off) * sm.Rd[o];
        const T e1 = sm.Es[(D - 1) * TC + u[D - 1] * (TE + 1)], d1 = sm.Ds[(D - 1) * TC + u[D - 1] * (TE + 1)];
        T pc = e1 * x;
        T gc = d1 * x;
        sm.Pin[(D - 2) * TD + o] = dev::fmadd(e1, x, P0s[D - 1]);
        sm.Gin[(D - 2) * TD + o] = dev::fmadd(d1, x, G0s[D - 1]);
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const T ep = sm.Es[l * TC + u[l] * (TE + 1)], dp = sm.Ds[l * TC + u[l] * (TE + 1)];
            gc = dev::fmadd(ep, gc, dp * pc);
            sm.Pin[(l - 1) * TD + o] = dev::fmadd(ep, pc, P0s[l]);
            sm.Gin[(l - 1) * TD + o] = G0s[l] + gc;
            pc = ep * pc;
        }
    }
    sm.Xs[o] = x;
    return isfinite(x) ? 0 : kErrNonfinite;
}

// Coupled groups of S members solved by one warp, 32 / S groups at a time:
// the warp's lanes form segments of S lanes, lane m of segment g holds the
// equation row of member m of group g.  Members are ordered with the 2x2
// modes of the group's `mask` as binary digits (member offset delta_mu(m) in
// {0, 1}).  Gaussian elimination with partial pivoting runs across the lanes
// of each segment with shuffles of width S; everything from outside the group
// is already in the running line sums Lin.  Packing the groups keeps the
// lanes of the FP64 pipes busy (a warp instruction occupies them whatever
// lanes are active).
__device__ __forceinline__ int member_delta(int mask, int m, int mu) {
    return ((mask >> mu) & 1) ? ((m >> __popc(mask & ((1 << mu) - 1))) & 1) : 0;
}
__device__ __forceinline__ int member_with(int mask, int m, int mu, int k) {
    if (!((mask >> mu) & 1)) return m;
    const int b = __popc(mask & ((1 << mu) - 1));
    return (m & ~(1 << b)) | (k << b);
}

template <typename T, int D, int FM, int S>
__device__ int warp_group_solve(const TileSmem<T, D, FM>& sm, const int* list, const int* moff, int count,
                                const T* Minv) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int TC = TE * TE;
    using C = WaveCfg<T, D, FM>;
    constexpr bool GEN = C::GEN;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane / S, m = lane % S;
    const bool act = g < count;
    // the lane's group: first element, 2x2 modes, precomputed inverse (if any)
    int a[D], mask = 0;
    {
        int rem = list[act ? g : 0] & 0xfff;
#pragma unroll
        for (int mu = 0; mu < D; mu++) {
            a[mu] = rem % TE;
            rem /= TE;
            if (sm.gl[mu * TE + sm.gidx[mu * TE + a[mu]]] == 2) mask |= 1 << mu;
        }
    }
    const int mo = moff[act ? g : 0];
    const T* minv = act && mo >= 0 ? Minv + mo : nullptr;
    int u[D], o = 0;
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        u[mu] = a[mu] + member_delta(mask, m, mu);
        o += u[mu] * ipow(TE, mu);
    }
    auto Dm = [&](int mu, int i, int k) -> T { return sm.Ds[mu * TC + i + TE * k]; };
    auto Em = [&](int mu, int i, int k) -> T { return sm.Es[mu * TC + i + TE * k]; };
    T r;
    T row[S];
    T P0[D], G0[D];
    if constexpr (C::TT) {
        // chain of the line sums through the group's diagonal blocks (other
        // members along each 2x2 mode), then the mode-1 level: c Q_1 + L_0
        P0[D - 1] = sm.Lin[C::slotP(D - 1) * TD + o];
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            T p = sm.Lin[C::slotP(l) * TD + o];
            const bool two = (mask >> l) & 1;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int src = member_with(mask, m, l, k);
                const T pp = dev::shfl(full, P0[l + 1], src, S);
                if (k == 0 || two) p = dev::fmadd(Em(l, u[l], two ? a[l] + k : u[l]), pp, p);
            }
            P0[l] = p;
        }
        T of = sm.Lin[(C::NACC - 1) * TD + o];
        {
            const bool two = mask & 1;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int src = member_with(mask, m, 0, k);
                const T pp = dev::shfl(full, P0[1], src, S);
                if (k == 0 || two) of = dev::fmadd(Em(0, u[0], two ? a[0] + k : u[0]), pp, of);
            }
        }
        r = sm.Rs[o] - of;
        // group system: A_1 (identity in the other modes) + C x A_2 x ... x A_d
#pragma unroll
        for (int k = 0; k < S; k++) {
            if (minv != nullptr) { row[k] = 0; continue; }
            bool same = true;
#pragma unroll
            for (int eta = 1; eta < D; eta++)
                if (member_delta(mask, m, eta) != member_delta(mask, k, eta)) same = false;
            T t = Em(0, u[0], a[0] + member_delta(mask, k, 0));
#pragma unroll
            for (int eta = 1; eta < D; eta++) t *= Em(eta, u[eta], a[eta] + member_delta(mask, k, eta));
            row[k] = same ? Dm(0, u[0], a[0] + member_delta(mask, k, 0)) + t : t;
        }
    } else if constexpr (!GEN) {
        r = sm.Rs[o] - sm.Lin[o];
#pragma unroll
        for (int k = 0; k < S; k++) {
            if (minv != nullptr) { row[k] = 0; continue; }
            T e = 0;
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                bool same = true;
#pragma unroll
                for (int eta = 0; eta < D; eta++)
                    if (eta != mu && member_delta(mask, m, eta) != member_delta(mask, k, eta)) same = false;
                if (same) e += Dm(mu, u[mu], a[mu] + member_delta(mask, k, mu));
            }
            row[k] = e;
        }
    } else {
        P0[D - 1] = sm.Lin[C::slotP(D - 1) * TD + o];
        G0[D - 1] = sm.Lin[C::slotG(D - 1) * TD + o];
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            T p = sm.Lin[C::slotP(l) * TD + o], q = sm.Lin[C::slotG(l) * TD + o];
            const bool two = (mask >> l) & 1;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int src = member_with(mask, m, l, k);
                const T pp = dev::shfl(full, P0[l + 1], src, S);
                const T gg = dev::shfl(full, G0[l + 1], src, S);
                if (k == 0 || two) {
                    const int kk = two ? a[l] + k : u[l];
                    p = dev::fmadd(Em(l, u[l], kk), pp, p);
                    q = dev::fmadd(Em(l, u[l], kk), gg, dev::fmadd(Dm(l, u[l], kk), pp, q));
                }
            }
            P0[l] = p;
            G0[l] = q;
        }
        T of = sm.Lin[(C::NACC - 1) * TD + o];
        {
            const bool two = mask & 1;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int src = member_with(mask, m, 0, k);
                const T pp = dev::shfl(full, P0[1], src, S);
                const T gg = dev::shfl(full, G0[1], src, S);
                if (k == 0 || two) {
                    const int kk = two ? a[0] + k : u[0];
                    of = dev::fmadd(Em(0, u[0], kk), gg, dev::fmadd(Dm(0, u[0], kk), pp, of));
                }
            }
        }
        r = sm.Rs[o] - of;
#pragma unroll
        for (int k = 0; k < S; k++) {
            if (minv != nullptr) { row[k] = 0; continue; }
            T e = 0;
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                const int v = a[mu] + member_delta(mask, k, mu);
                T t = Dm(mu, u[mu], v);
#pragma unroll
                for (int eta = 0; eta < D; eta++)
                    if (eta != mu) t *= Em(eta, u[eta], a[eta] + member_delta(mask, k, eta));
                e += t;
            }
            row[k] = e;
        }
    }
    // lanes of a group that is not eliminated here (it has an inverse, or the
    // segment has no group) carry an identity row, which the elimination
    // leaves as it is
    const bool ge = act && minv == nullptr;
    if (!act) r = 0;
    if (!ge) {
#pragma unroll
        for (int k = 0; k < S; k++) row[k] = k == m ? T(1) : T(0);
    }
    int status = 0;
    T x = 0;
    if (__any_sync(full, minv != nullptr)) {
        // precomputed inverse: x_m = sum_k Minv(m, k) r_k
#pragma unroll
        for (int k = 0; k < S; k++) {
            const T rk = dev::shfl(full, r, k, S);
            if (minv != nullptr) x = dev::fmadd(minv[m * S + k], rk, x);
        }
        x = dev::settle(x);
    }
    if (__any_sync(full, ge)) {
        // scale for the pivot test: 16 eps max |M| over the group (magnitudes
        // in the real type of T)
        using R = typename RealOf<T>::type;
        R big = 0;
#pragma unroll
        for (int k = 0; k < S; k++) big = fmax(big, fabs(row[k]));
#pragma unroll
        for (int w = S / 2; w >= 1; w >>= 1) big = fmax(big, __shfl_xor_sync(full, big, w, S));
        const R tiny = R(16) * dev::Eps<T>::v * big;
        // forward elimination; the reciprocal of each pivot stays with the
        // pivot's lane for the back substitution
        T dinv = T(1);
#pragma unroll
        for (int c = 0; c < S; c++) {
            R val = m >= c ? fabs(row[c]) : R(-1);
            int idx = m;
#pragma unroll
            for (int w = S / 2; w >= 1; w >>= 1) {
                const R ov = __shfl_xor_sync(full, val, w, S);
                const int oi = __shfl_xor_sync(full, idx, w, S);
                if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
            }
            const int pv = idx;  // identical on the lanes of a segment
            if (__any_sync(full, pv != c)) {
                const int src = m == c ? pv : (m == pv ? c : m);
#pragma unroll
                for (int k = 0; k < S; k++) row[k] = dev::shfl(full, row[k], src, S);
                r = dev::shfl(full, r, src, S);
            }
            // the pivot row is broadcast one entry at a time
            const T pc = dev::shfl(full, row[c], c, S);
            if (ge && !(fabs(pc) > tiny)) status |= kErrSingular;
            const T rinv = T(1) / pc;
            if (m == c) dinv = rinv;
            const T f = row[c] * rinv;
            // (double-float: the updated pairs are normalised, so that the
            // pivot tests, which read the high word, see their value after
            // the cancellation that elimination is made of)
#pragma unroll
            for (int k = c + 1; k < S; k++) {
                const T pk = dev::shfl(full, row[k], c, S);
                if (m > c) row[k] = dev::settle(dev::fmadd(-f, pk, row[k]));
            }
            const T pr = dev::shfl(full, r, c, S);
            if (m > c) r = dev::settle(dev::fmadd(-f, pr, r));
        }
        // back substitution; lane m ends with x_m
#pragma unroll
        for (int c = S - 1; c >= 0; c--) {
            const T xc = dev::shfl(full, r * dinv, c, S);
            if (ge && m == c) x = xc;
            if (m < c) r = dev::settle(dev::fmadd(-row[c], xc, r));
        }
    }
    if (act) {
        if (!isfinite(x)) status |= kErrNonfinite;
        sm.Xs[o] = x;
    }
    if constexpr (C::TT) {
        // completion of the in-block intermediates Q_l at the group positions
        T pc[D];
        {
            constexpr int mu = D - 1;
            const bool two = (mask >> mu) & 1;
            T p = 0;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const T xv = dev::shfl(full, x, member_with(mask, m, mu, k), S);
                if (k == 0 || two) p = dev::fmadd(Em(mu, u[mu], two ? a[mu] + k : u[mu]), xv, p);
            }
            pc[mu] = p;
        }
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const bool two = (mask >> l) & 1;
            T p = 0;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const T pp = dev::shfl(full, pc[l + 1], member_with(mask, m, l, k), S);
                if (k == 0 || two) p = dev::fmadd(Em(l, u[l], two ? a[l] + k : u[l]), pp, p);
            }
            pc[l] = p;
        }
        if (act) {
#pragma unroll
            for (int l = 1; l < D; l++) sm.Pin[(l - 1) * TD + o] = P0[l] + pc[l];
        }
    }
    if constexpr (GEN) {
        // completion of the in-block intermediates at the group positions
        T pc[D], gc[D];
        {
            constexpr int mu = D - 1;
            const bool two = (mask >> mu) & 1;
            T p = 0, q = 0;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const T xv = dev::shfl(full, x, member_with(mask, m, mu, k), S);
                if (k == 0 || two) {
                    const int kk = two ? a[mu] + k : u[mu];
                    p = dev::fmadd(Em(mu, u[mu], kk), xv, p);
                    q = dev::fmadd(Dm(mu, u[mu], kk), xv, q);
                }
            }
            pc[mu] = p;
            gc[mu] = q;
        }
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const bool two = (mask >> l) & 1;
            T p = 0, q = 0;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int src = member_with(mask, m, l, k);
                const T pp = dev::shfl(full, pc[l + 1], src, S);
                const T gg = dev::shfl(full, gc[l + 1], src, S);
                if (k == 0 || two) {
                    const int kk = two ? a[l] + k : u[l];
                    p = dev::fmadd(Em(l, u[l], kk), pp, p);
                    q = dev::fmadd(Em(l, u[l], kk), gg, dev::fmadd(Dm(l, u[l], kk), pp, q));
                }
            }
            pc[l] = p;
            gc[l] = q;
        }
        if (act) {
#pragma unroll
            for (int l = 1; l < D; l++) {
                sm.Pin[(l - 1) * TD + o] = P0[l] + pc[l];
                sm.Gin[(l - 1) * TD + o] = G0[l] + gc[l];
            }
        }
    }
    return status;
}

// Warp-uniform entry: `count` (<= 32 >> cls) groups with cls coupled modes,
// listed at `list` (first in-block element of each) with their inverse
// offsets at `moff` (-1: none).
template <typename T, int D, int FM>
__device__ int warp_group(const TileSmem<T, D, FM>& sm, int cls, const int* list, const int* moff, int count,
                          const T* Minv) {
    switch (cls) {
        case 1: return warp_group_solve<T, D, FM, 2>(sm, list, moff, count, Minv);
        case 2: return warp_group_solve<T, D, FM, 4>(sm, list, moff, count, Minv);
        case 3: if constexpr (D >= 3) return warp_group_solve<T, D, FM, 8>(sm, list, moff, count, Minv); else return 0;
        case 4: if constexpr (D >= 4) return warp_group_solve<T, D, FM, 16>(sm, list, moff, count, Minv); else return 0;
        case 5: if constexpr (D >= 5) return warp_group_solve<T, D, FM, 32>(sm, list, moff, count, Minv); else return 0;
        default: return 0;
    }
}

// Running line sums of element e (owned by this thread) when its
// anti-diagonal comes: along every mode, the products of the diagonal-block
// coefficients with the solved positions beyond e's group (the solution X for
// the Laplace form; X, P_{l+1}, G_{l+1} for the levels of the generalized
// recurrence).  The modes are independent and each sum runs as two
// interleaved chains, so the latency is that of a few multiply-adds.
template <typename T, int D, int FM>
__device__ __forceinline__ void pull_lines(const TileSmem<T, D, FM>& sm, int e, const int (&u)[D], const int (&k0s)[D],
                                           T (&L)[WaveCfg<T, D, FM>::NACC], bool on) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int TC = TE * TE;
    using C = WaveCfg<T, D, FM>;
    constexpr bool GEN = C::GEN;
    const T* __restrict__ Xs = sm.Xs;
    T lap[D];
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        const int st = ipow(TE, mu);
        const int k0 = k0s[mu];  // first index beyond e's group along mode mu
        const int kb = sm.bs[mu];
        T a0 = 0, a1 = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0;
        // FP32: all TE terms with the coefficients before k0 masked to zero
        // (positions beyond the block extent hold zeros), fully unrolled so
        // that every load is in flight at once; wider types: only the terms
        // needed (the FP64 pipe is the scarce resource there, and a warp
        // instruction occupies it whatever lanes are active).  WARP_TERMS:
        // the range starts at the warp's first needed term (`on` marks the
        // lanes that hold an element; all 32 lanes call).
        constexpr bool FULL = sizeof(T) == 4;
        constexpr bool WT = C::WARP_TERMS;
        int wlo = 0;
        if constexpr (WT) wlo = __reduce_min_sync(0xffffffffu, on ? k0 : TE);
#pragma unroll
        for (int kk = 0; kk < TE; kk++) {
            const int k = WT ? wlo + kk : kk;
            if (WT && k >= kb) break;  // uniform over the warp
            if (!FULL && (k < k0 || k >= kb)) continue;
            const bool in = !FULL || k >= k0;
            const int v = in ? e + (k - u[mu]) * st : e;
            const T dv = in ? sm.Ds[mu * TC + u[mu] + TE * k] : T(0);
            const bool odd = kk & 1;
            if constexpr (C::TT) {
                // chain factor (C in mode 1, A_mu elsewhere) on X (mode d) or
                // on Q_{mu+1}; mode 1 also carries A_1 on X
                const T ev = in ? sm.Es[mu * TC + u[mu] + TE * k] : T(0);
                if (mu == D - 1) {
                    const T xv = in ? Xs[v] : T(0);
                    if (odd) a1 = dev::fmadd(ev, xv, a1); else a0 = dev::fmadd(ev, xv, a0);
                } else if (mu >= 1) {
                    const T pv = in ? sm.Pin[mu * TD + v] : T(0);  // level mu + 1
                    if (odd) a1 = dev::fmadd(ev, pv, a1); else a0 = dev::fmadd(ev, pv, a0);
                } else {
                    const T pv = in ? sm.Pin[v] : T(0), xv = in ? Xs[v] : T(0);  // level 1
                    if (odd) { a1 = dev::fmadd(ev, pv, a1); b1 = dev::fmadd(dv, xv, b1); }
                    else { a0 = dev::fmadd(ev, pv, a0); b0 = dev::fmadd(dv, xv, b0); }
                }
            } else if constexpr (!GEN) {
                const T xv = in ? Xs[v] : T(0);
                if (odd) a1 = dev::fmadd(dv, xv, a1); else a0 = dev::fmadd(dv, xv, a0);
            } else {
                const T ev = in ? sm.Es[mu * TC + u[mu] + TE * k] : T(0);
                if (mu == D - 1) {
                    const T xv = in ? Xs[v] : T(0);
                    if (odd) { a1 = dev::fmadd(ev, xv, a1); b1 = dev::fmadd(dv, xv, b1); }
                    else { a0 = dev::fmadd(ev, xv, a0); b0 = dev::fmadd(dv, xv, b0); }
                } else if (mu >= 1) {
                    const T pv = in ? sm.Pin[mu * TD + v] : T(0), gv = in ? sm.Gin[mu * TD + v] : T(0);  // level mu + 1
                    if (odd) { a1 = dev::fmadd(ev, pv, a1); b1 = dev::fmadd(ev, gv, b1); c1 = dev::fmadd(dv, pv, c1); }
                    else { a0 = dev::fmadd(ev, pv, a0); b0 = dev::fmadd(ev, gv, b0); c0 = dev::fmadd(dv, pv, c0); }
                } else {
                    const T pv = in ? sm.Pin[v] : T(0), gv = in ? sm.Gin[v] : T(0);                       // level 1
                    if (odd) { a1 = dev::fmadd(ev, gv, a1); b1 = dev::fmadd(dv, pv, b1); }
                    else { a0 = dev::fmadd(ev, gv, a0); b0 = dev::fmadd(dv, pv, b0); }
                }
            }
        }
        if constexpr (C::TT) {
            if (mu >= 1) L[C::slotP(mu)] = a0 + a1;
            else L[C::NACC - 1] = (a0 + a1) + (b0 + b1);
        } else if constexpr (!GEN) {
            lap[mu] = a0 + a1;
        } else {
            if (mu == D - 1) {
                L[C::slotP(D - 1)] = a0 + a1;
                L[C::slotG(D - 1)] = b0 + b1;
            } else if (mu >= 1) {
                L[C::slotP(mu)] = a0 + a1;
                L[C::slotG(mu)] = (b0 + b1) + (c0 + c1);
            } else {
                L[C::NACC - 1] = (a0 + a1) + (b0 + b1);
            }
        }
    }
    if constexpr (!GEN && !C::TT) {
        T sum = lap[0];
#pragma unroll
        for (int mu = 1; mu < D; mu++) sum += lap[mu];
        L[0] = sum;
    }
}

// Entry (m, k) of the system of a coupled group with first element a and 2x2
// modes `mask`: the operator restricted to the group (Laplace: the Kronecker
// sum of the diagonal blocks; generalized: sum_mu A_mu x prod_{eta!=mu} C_eta).
template <typename T, int D, int FM>
__device__ __forceinline__ T group_entry(const TileSmem<T, D, FM>& sm, const int (&a)[D], int mask, int m, int k) {
    constexpr int TE = tile_extent(D);
    constexpr int TC = TE * TE;
    constexpr bool GEN = WaveCfg<T, D, FM>::GEN;
    if constexpr (WaveCfg<T, D, FM>::TT) {
        // A_1 (identity in the other modes) + C x A_2 x ... x A_d on the group
        bool same = true;
        T t = 1;
#pragma unroll
        for (int mu = 0; mu < D; mu++) {
            const int i = a[mu] + member_delta(mask, m, mu), j = a[mu] + member_delta(mask, k, mu);
            t *= sm.Es[mu * TC + i + TE * j];
            if (mu >= 1 && i != j) same = false;
        }
        const int i0 = a[0] + member_delta(mask, m, 0), j0 = a[0] + member_delta(mask, k, 0);
        return same ? sm.Ds[i0 + TE * j0] + t : t;
    }
    T e = 0;
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        const int i = a[mu] + member_delta(mask, m, mu), j = a[mu] + member_delta(mask, k, mu);
        T t = sm.Ds[mu * TC + i + TE * j];
#pragma unroll
        for (int eta = 0; eta < D; eta++) {
            if (eta == mu) continue;
            const int ii = a[eta] + member_delta(mask, m, eta), jj = a[eta] + member_delta(mask, k, eta);
            if constexpr (GEN) t *= sm.Es[eta * TC + ii + TE * jj];
            else if (ii != jj) t = T(0);
        }
        e += t;
    }
    return e;
}

// Inverse of a coupled group's system (S x S, row-major into out), by
// Gauss-Jordan elimination with partial pivoting.  Returns kErrSingular for a
// pivot below 16 eps max|M|.
template <typename T, int D, int GEN, int S>
__device__ int group_inverse_s(const TileSmem<T, D, GEN>& sm, const int (&a)[D], int mask, T* out) {
    T W[S][2 * S];
    using R = typename RealOf<T>::type;
    R big = 0;
#pragma unroll
    for (int m = 0; m < S; m++)
#pragma unroll
        for (int k = 0; k < S; k++) {
            W[m][k] = group_entry<T, D, GEN>(sm, a, mask, m, k);
            W[m][S + k] = m == k ? T(1) : T(0);
            big = fmax(big, fabs(W[m][k]));
        }
    const R tiny = R(16) * dev::Eps<T>::v * big;
    int status = 0;
#pragma unroll
    for (int c = 0; c < S; c++) {
#pragma unroll
        for (int q = c + 1; q < S; q++) {
            const bool sw = fabs(W[q][c]) > fabs(W[c][c]);
#pragma unroll
            for (int k = 0; k < 2 * S; k++) {
                const T x = W[c][k], y = W[q][k];
                W[c][k] = sw ? y : x;
                W[q][k] = sw ? x : y;
            }
        }
        if (!(fabs(W[c][c]) > tiny)) status |= kErrSingular;
        const T inv = T(1) / W[c][c];
#pragma unroll
        for (int k = 0; k < 2 * S; k++) W[c][k] *= inv;
#pragma unroll
        for (int q = 0; q < S; q++) {
            if (q == c) continue;
            const T f = W[q][c];
#pragma unroll
            for (int k = 0; k < 2 * S; k++) W[q][k] = dev::settle(dev::fmadd(-f, W[c][k], W[q][k]));
        }
    }
#pragma unroll
    for (int m = 0; m < S; m++)
#pragma unroll
        for (int k = 0; k < S; k++) out[m * S + k] = W[m][S + k];
    return status;
}

template <typename T, int D, int GEN>
__device__ int group_inverse(const TileSmem<T, D, GEN>& sm, int e, T* out) {
    constexpr int TE = tile_extent(D);
    int a[D], mask = 0, rem = e;
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        a[mu] = rem % TE;
        rem /= TE;
        if (sm.gl[mu * TE + sm.gidx[mu * TE + a[mu]]] == 2) mask |= 1 << mu;
    }
    switch (__popc(mask)) {
        case 1: return group_inverse_s<T, D, GEN, 2>(sm, a, mask, out);
        case 2: return group_inverse_s<T, D, GEN, 4>(sm, a, mask, out);
        default: return 0;  // larger groups are eliminated in place by a warp
    }
}

// One block T of the block grid: its right-hand-side update (split over the
// `csize` CTAs of a cluster, this CTA being `rank`) and, on rank 0, its base
// case.  The CTA's NST staging barriers `bar` are initialised by the caller;
// uses[s] counts the phases barrier s has completed so far (a persistent
// caller runs many blocks on the same barriers).  Returns false when a wait
// ran out of time (the error word is set; no copy of this call is left in
// flight).
// PK selects the arithmetic of the block updates: the native FMA pipes, or
// (FP32 solves only) TF32 / BF16 tensor-core products with FP32 accumulation.
template <typename T, int D, int GENF, int PK = kProdNative>
__device__ __forceinline__ bool wave_tile(const WaveArgs& a, const long long t, const int rank, const int csize,
                                          uint32_t (&uses)[WaveCfg<T, D, GENF>::NST], uint64_t* bar) {
    using C = WaveCfg<T, D, GENF>;
    constexpr int TE = C::TE, TD = C::TD, TC = C::TC, EPT = C::EPT, NACC = C::NACC;
    constexpr bool GEN = C::GEN, TT = C::TT, CHAIN = C::CHAIN;
    constexpr bool TCU = PK != kProdNative;  // tensor-core updates
    static_assert(!TCU || (PK == kProdDMMA ? sizeof(T) == 8 && !IsComplex<T>::value : sizeof(T) == 4),
                  "TF32 / BF16 tensor-core block updates serve the FP32 solve, DMMA the FP64 solve");
    using Q = MmaCfg<D, TCU ? PK : kProdTF32>;
    using QF = typename Q::F;
    constexpr int NS = GEN ? NACC : D;        // accumulator slots of the fragments
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sbase = reinterpret_cast<T*>(smem_raw);
    T* stage = sbase + C::oStage;
    T* red = sbase + C::oRed;
    int* meta = reinterpret_cast<int*>(smem_raw + C::oMeta);
    int* gs = meta;                  // [D][TE]
    int* gl = gs + D * TE;           // [D][TE]
    int* ng = gl + D * TE;           // [D]
    int* bs = ng + D;                // [D]

    const int tid = threadIdx.x;
    int I[D];
#pragma unroll
    for (int mu = 0; mu < D; mu++) I[mu] = static_cast<int>((t / a.tstride[mu]) % a.nb[mu]);

    // ---- job list: level L covers mode L (Laplace) or d-1-L (generalized).
    // Jobs run in decreasing distance dd = J' - I_mu of the source block
    // (levels in order within one distance): in a persistent launch the
    // nearest source blocks are the last ones to be solved.
    int cnt[D], w[D], maxc = 0;
    long long W = 0;
#pragma unroll
    for (int L = 0; L < D; L++) {
        const int mu = CHAIN ? D - 1 - L : L;
        cnt[L] = a.hi[mu] - 1 - I[mu];
        if (cnt[L] < 0) cnt[L] = 0;
        if (cnt[L] > maxc) maxc = cnt[L];
        w[L] = GEN ? ((L == 0 || L == D - 1) ? 2 : 3) : TT ? (L == D - 1 ? 2 : 1) : 1;
        W += static_cast<long long>(cnt[L]) * w[L];
    }
    // number of jobs whose distance is at least dd
    auto at_least = [&](int dd) {
        int n = 0;
#pragma unroll
        for (int L = 0; L < D; L++) n += cnt[L] >= dd ? cnt[L] - dd + 1 : 0;
        return n;
    };
    const int jt = at_least(1);
    int j0 = 0, j1 = jt;
    if (csize > 1) {
        // split the jobs over the cluster by weight, in job order
        const long long wlo = W * rank / csize, whi = W * (rank + 1) / csize;
        long long cw = 0;
        int j = 0;
        bool f0 = false, f1 = false;
        for (int dd = maxc; dd >= 1; dd--)
            for (int L = 0; L < D; L++) {
                if (cnt[L] < dd) continue;
                if (!f0 && cw >= wlo) { j0 = j; f0 = true; }
                if (!f1 && cw >= whi) { j1 = j; f1 = true; }
                cw += w[L];
                j++;
            }
        if (!f0) j0 = jt;
        if (!f1) j1 = jt;
    }
    const int njob = j1 - j0;

    // job j -> (level, source block J')
    auto decode = [&](int j, int& L, int& Jp) {
        int lo = 1, hi = maxc;  // largest dd with at_least(dd) > j
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (at_least(mid) > j) lo = mid; else hi = mid - 1;
        }
        int r = j - at_least(lo + 1);
        L = 0;
        for (int q = 0; q < D; q++) {
            if (cnt[q] < lo) continue;
            if (r == 0) { L = q; break; }
            r--;
        }
        const int mu = CHAIN ? D - 1 - L : L;
        Jp = I[mu] + lo;
    };
    int* jtab = reinterpret_cast<int*>(smem_raw + C::oJob);
    unsigned* jready = reinterpret_cast<unsigned*>(jtab + C::JT);
    auto job = [&](int j, int& L, int& Jp) {
        const int r = j - j0;
        if (r < C::JT) {
            const int v = jtab[r];
            L = v >> 24;
            Jp = v & 0xffffff;
        } else {
            decode(j, L, Jp);
        }
    };
    auto issue = [&](int j, int stg) {
        int L, Jp;
        job(j, L, Jp);
        const int mu = CHAIN ? D - 1 - L : L;
        const long long ts = t + static_cast<long long>(Jp - I[mu]) * a.tstride[mu];
        const long long tri = static_cast<long long>(Jp) * (Jp + 1) / 2 + I[mu];
        T* sb = stage + stg * C::STAGE;
        const T* S1;
        const T* S2 = nullptr;
        const T* M1;
        const T* M2 = nullptr;
        if (TT) {
            // two-term form: Q_{mu+1} x A_mu (Q_d = X); mode 1: Q_1 x C + X x A_1
            if (mu >= 1) {
                S1 = static_cast<const T*>(L == 0 ? a.X : a.P[mu + 1]) + ts * TD;
                M1 = static_cast<const T*>(a.At[mu]) + tri * TC;
            } else {
                S1 = static_cast<const T*>(a.X) + ts * TD;
                S2 = static_cast<const T*>(D >= 2 ? a.P[1] : a.X) + ts * TD;
                M1 = static_cast<const T*>(a.Ct[0]) + tri * TC;
                M2 = static_cast<const T*>(a.At[0]) + tri * TC;
            }
        } else if (!GEN) {
            S1 = static_cast<const T*>(a.X) + ts * TD;
            M1 = static_cast<const T*>(a.At[mu]) + tri * TC;
        } else {
            if (L == 0) {
                S1 = static_cast<const T*>(a.X) + ts * TD;
            } else {
                S1 = static_cast<const T*>(a.P[mu + 1]) + ts * TD;
                S2 = static_cast<const T*>(a.G[mu + 1]) + ts * TD;
            }
            M1 = static_cast<const T*>(a.Ct[mu]) + tri * TC;
            M2 = static_cast<const T*>(a.At[mu]) + tri * TC;
        }
        const int r = j - j0;
        if (a.ready && !(r < C::JT && ((jready[r >> 5] >> (r & 31)) & 1u))) {
            // persistent launch: the source block must be solved (bounded wait)
            if (!dev::wait_at_least(a.ready + ts, 1, a.abort, a.timeout_ns)) atomicOr(a.err, kErrTimeout);
            dev::fence_proxy_async_all();
        }
        const uint32_t bytes = static_cast<uint32_t>(((S2 ? 2 : 1) * TD + (M2 ? 2 : 1) * TC) * sizeof(T));
        dev::mbar_expect_tx(&bar[stg], bytes);
        dev::bulk_g2s(sb, S1, TD * sizeof(T), &bar[stg]);
        if (S2) dev::bulk_g2s(sb + TD, S2, TD * sizeof(T), &bar[stg]);
        dev::bulk_g2s(sb + 2 * TD, M1, TC * sizeof(T), &bar[stg]);
        if (M2) dev::bulk_g2s(sb + 2 * TD + TC, M2, TC * sizeof(T), &bar[stg]);
    };

    T acc[NACC][EPT];
#pragma unroll
    for (int s = 0; s < NACC; s++)
#pragma unroll
        for (int q = 0; q < EPT; q++) acc[s][q] = T(0);
    QF cfr[TCU ? NS : 1][TCU ? Q::UPW : 1][Q::NF];
    if constexpr (TCU) {
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int u = 0; u < Q::UPW; u++)
#pragma unroll
                for (int h = 0; h < 4; h++) cfr[s][u][h] = 0.f;
    }

    constexpr int NST = C::NST;
    // decode the first JT jobs and, in a persistent launch, test their source
    // blocks' flags, one job per thread (one round trip instead of one per job)
    {
        const int r = tid;
        bool rdy = false;
        if (r < C::JT && r < njob) {
            int L, Jp;
            decode(j0 + r, L, Jp);
            jtab[r] = (L << 24) | Jp;
            if (a.ready) {
                const int mu = CHAIN ? D - 1 - L : L;
                rdy = dev::ld_acquire(a.ready + t + static_cast<long long>(Jp - I[mu]) * a.tstride[mu]) != 0;
            }
        }
        const unsigned bits = __ballot_sync(0xffffffffu, rdy);
        if ((tid & 31) == 0 && tid < C::JT) jready[tid >> 5] = bits;
        __syncthreads();
    }
    if (tid == 0) {
        dev::fence_proxy_async_all();
        for (int q = 0; q < NST && q < njob; q++) issue(j0 + q, q);
    }
    // ---- base case of block T, the part that depends only on the diagonal
    // blocks of the coefficients (done while the first copies are in flight,
    // so that only the rest follows the wait for the nearest source blocks):
    // diagonal tiles, right-hand side, 2x2 group structure, reciprocal
    // diagonal, the anti-diagonal buckets and the coupled-group list
    T* Rs = sbase + C::oR;
    T* Xs = sbase + C::oX;
    T* Rd = sbase + C::oRd;
    T* Pin = sbase + C::oPin;
    T* Gin = sbase + C::oGin;
    T* Ds = sbase + C::oD;
    T* Es = sbase + C::oE;
    T* Lin = sbase + C::oLin;
    int* gidx = bs + D + 4;          // [D][TE] group of every in-block index
    T* Xg = static_cast<T*>(a.X) + t * TD;
    for (int idx = tid; idx < D * TC; idx += kThreads) {
        const int mu = idx / TC, e = idx % TC;
        const long long tri = static_cast<long long>(I[mu]) * (I[mu] + 1) / 2 + I[mu];
        Ds[idx] = static_cast<const T*>(a.At[mu])[tri * TC + e];
        if (GEN) Es[idx] = static_cast<const T*>(a.Ct[mu])[tri * TC + e];
        // two-term form: the chain factor of every mode (C in mode 1, A_mu elsewhere)
        if (TT) Es[idx] = static_cast<const T*>(mu == 0 ? a.Ct[0] : a.At[mu])[tri * TC + e];
    }
    for (int e = tid; e < TD; e += kThreads) {
        Rs[e] = Xg[e];
        Xs[e] = T(0);
    }
    int* cg_cnt = gidx + D * TE;        // coupled groups per anti-diagonal
    int* cg_off = cg_cnt + C::MAXSTEP;  // their offsets in cg_list
    int* cg_fill = cg_off + C::MAXSTEP + 1;
    int* cg_list = cg_fill + C::MAXSTEP;  // class << 12 | first element (in-block elements < 4096)
    int* cg_moff = cg_list + (TD / 2 + 1);  // offset of each group's inverse (-1: none)
    int* act_cnt = cg_moff + (TD / 2 + 1);  // elements per anti-diagonal
    int* act_off = act_cnt + C::MAXSTEP;
    int* act_fill = act_off + C::MAXSTEP + 1;
    int* act_list = act_fill + C::MAXSTEP;  // element codes (ElemCode)
    T* Minv = sbase + C::oMinv;
    for (int i = tid; i < C::MAXSTEP; i += kThreads) { cg_cnt[i] = 0; cg_fill[i] = 0; act_cnt[i] = 0; act_fill[i] = 0; }
    if (CHAIN && !C::PIN_IN_RING)
        for (int e = tid; e < C::NL * TD; e += kThreads) { Pin[e] = T(0); Gin[e] = T(0); }
    if (tid < D) bs[tid] = a.bsize[tid][I[tid]];
    __syncthreads();
    if (tid < D) {
        const int mu = tid, b = bs[mu];
        int n = 0, i = 0;
        while (i < b) {
            if (!C::CPLX && i + 1 < b && Ds[mu * TC + (i + 1) + TE * i] != T(0)) {
                gs[mu * TE + n] = i; gl[mu * TE + n] = 2;
                gidx[mu * TE + i] = n; gidx[mu * TE + i + 1] = n;
                i += 2;
            } else {
                gs[mu * TE + n] = i; gl[mu * TE + n] = 1;
                gidx[mu * TE + i] = n;
                i += 1;
            }
            n++;
        }
        for (int k = b; k < TE; k++) gidx[mu * TE + k] = 0;
        ng[mu] = n;
    }
    __syncthreads();  // the group tables are read by every thread below
    // Every thread owns the elements e = tid + q*kThreads: it solves those
    // that are 1x1 groups (or leads a coupled group) when their anti-diagonal
    // comes.
    int status = 0;
    int uq[EPT][D], gq[EPT][D], sq[EPT];
    bool okq[EPT], lead[EPT], single[EPT];
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = tid + q * kThreads;
        okq[q] = (TD % kThreads) == 0 || e < TD;
        int rem = e, sgv = 0, S = 1;
        bool ld = true;
#pragma unroll
        for (int mu = 0; mu < D; mu++) {
            const int i = rem % TE;
            rem /= TE;
            uq[q][mu] = i;
            if (i >= bs[mu]) okq[q] = false;
            const int gg = okq[q] ? gidx[mu * TE + i] : 0;
            gq[q][mu] = gg;
            sgv += gg;
            if (okq[q]) {
                S *= gl[mu * TE + gg];
                if (gs[mu * TE + gg] != i) ld = false;
            }
        }
        sq[q] = sgv;
        single[q] = okq[q] && S == 1;
        lead[q] = okq[q] && S > 1 && ld;
        if (single[q] && TT) {
            // two-term form: a_1,ii + c_ii prod_{mu >= 2} a_mu,jj
            T t2 = Es[uq[q][0] * (TE + 1)];
#pragma unroll
            for (int mu = 1; mu < D; mu++) t2 *= Es[mu * TC + uq[q][mu] * (TE + 1)];
            const T t1 = Ds[uq[q][0] * (TE + 1)];
            const T diag = dev::add_rn(t1, t2);  // never fused with the product above
            if (!(fabs(diag) > typename RealOf<T>::type(16) * dev::Eps<T>::v * (fabs(t1) + fabs(t2))))
                status |= kErrSingular;
            Rd[e] = T(1) / diag;
        } else if (single[q]) {
            // reciprocal of the diagonal entry sum_mu a_mu,ii prod_{eta != mu} c_eta,jj
            T diag = 0;
            typename RealOf<T>::type mag = 0;
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                T tt = Ds[mu * TC + uq[q][mu] * (TE + 1)];
                if constexpr (GEN) {
#pragma unroll
                    for (int eta = 0; eta < D; eta++)
                        if (eta != mu) tt *= Es[eta * TC + uq[q][eta] * (TE + 1)];
                }
                diag = dev::add_rn(diag, tt);  // never fused with the product above
                mag += fabs(tt);
            }
            if (!(fabs(diag) > typename RealOf<T>::type(16) * dev::Eps<T>::v * mag)) status |= kErrSingular;
            Rd[e] = T(1) / diag;
        }
    }
    // element slots of the block updates whose whole warp holds padding only
    unsigned live = 0;
#pragma unroll
    for (int q = 0; q < EPT; q++)
        if (__ballot_sync(0xffffffffu, okq[q])) live |= 1u << q;
    // the tensor-core variant's output tiles that hold padding only
    const unsigned tlive = TCU ? mma_tile_live<D, TCU ? PK : kProdTF32>(bs) : 0u;
    int nsum = 0;
#pragma unroll
    for (int mu = 0; mu < D; mu++) nsum += ng[mu];
    // coupled groups, bucketed by anti-diagonal (solved one warp per group)
    // and all elements, bucketed the same way (each anti-diagonal's elements
    // are handled by the first threads, so idle warps issue nothing)
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        if (lead[q]) atomicAdd(&cg_cnt[sq[q]], 1);
        if (okq[q]) atomicAdd(&act_cnt[sq[q]], 1);
    }
    __syncthreads();
    if (tid == 0) {
        cg_off[0] = 0;
        for (int i = 0; i < C::MAXSTEP; i++) cg_off[i + 1] = cg_off[i] + cg_cnt[i];
    } else if (tid == 32) {
        act_off[0] = 0;
        for (int i = 0; i < C::MAXSTEP; i++) act_off[i + 1] = act_off[i] + act_cnt[i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        if (lead[q]) cg_list[cg_off[sq[q]] + atomicAdd(&cg_fill[sq[q]], 1)] = tid + q * kThreads;
        if (okq[q])
            act_list[act_off[sq[q]] + atomicAdd(&act_fill[sq[q]], 1)] = ElemCode<D>::make(
                tid + q * kThreads, !single[q], [&](int mu) { return gs[mu * TE + gq[q][mu]] + gl[mu * TE + gq[q][mu]]; });
    }
    __syncthreads();
    // inverses of the coupled groups with <= 4 members (the system depends only
    // on the diagonal blocks), all groups in parallel: here when they have a
    // region of their own, else after the block updates (in the staging ring)
    const int ncg = cg_off[C::MAXSTEP];
    if (tid == 0) {
        // canonical order within every anti-diagonal (the fill order above
        // depends on the atomics), so that which groups get an inverse within
        // the budget, and hence the rounding, is the same in every run: by
        // class (number of coupled modes), then by first element, so that
        // the groups of one class that a warp solves together are adjacent
        auto cls_of = [&](int e) {
            int rem = e, mask = 0;
            for (int mu = 0; mu < D; mu++) {
                const int ai = rem % TE;
                rem /= TE;
                if (gl[mu * TE + gidx[mu * TE + ai]] == 2) mask |= 1 << mu;
            }
            return __popc(mask);
        };
        for (int st = 0; st < C::MAXSTEP; st++)
            for (int i = cg_off[st]; i < cg_off[st + 1]; i++) {
                const int v = (cls_of(cg_list[i]) << 12) | cg_list[i];
                int k = i - 1;
                for (; k >= cg_off[st] && cg_list[k] > v; k--) cg_list[k + 1] = cg_list[k];
                cg_list[k + 1] = v;
            }
        int run = 0;
        for (int i = 0; i < ncg; i++) {
            const int S = 1 << (cg_list[i] >> 12);
            if (S <= 4 && run + S * S <= C::MINV) {
                cg_moff[i] = run;
                run += S * S;
            } else {
                cg_moff[i] = -1;
            }
        }
    }
    __syncthreads();
    if constexpr (C::INV_EARLY) {
        const TileSmem<T, D, GENF> smi{Ds, Es, Rs, Rd, Xs, Pin, Gin, Lin, gs, gl, ng, bs, gidx};
        for (int i = tid; i < ncg; i += kThreads)
            if constexpr (!C::CPLX)
                if (cg_moff[i] >= 0) status |= group_inverse<T, D, GENF>(smi, cg_list[i] & 0xfff, Minv + cg_moff[i]);
    }
    bool dead = false;
    for (int jj = 0; jj < njob && !dead; jj++) {
        const int stg = jj % NST;
        // uniform over the warp (the tensor-core variants issue warp-wide mma)
        const bool ok = __all_sync(0xffffffffu, dev::mbar_wait(&bar[stg], (uses[stg] + static_cast<uint32_t>(jj / NST)) & 1u,
                                                               a.timeout_ns));
        if (ok) {  // a warp whose wait ran out skips the job; the block is abandoned below
            int L, Jp;
            job(j0 + jj, L, Jp);
            // padding skipped where the FP64 pipes bound the updates (FP64,
            // complex); the latency-bound FP32 updates run full tiles
            const int ks = sizeof(T) >= 8 ? a.bsize[CHAIN ? D - 1 - L : L][Jp] : TE;
            if constexpr (TCU)
                mma_dispatch<D, GEN, PK, NS>(L, cfr, reinterpret_cast<const QF*>(stage + stg * C::STAGE), ks, tlive);
            else
                dispatch_job<T, D, GENF>(L, acc, stage + stg * C::STAGE, ks, sizeof(T) >= 8 ? live : ~0u);
        }
        // one barrier per job: every thread is done reading the stage (it
        // orders those reads before the copies that refill it, as for a
        // consumer-release mbarrier arrival), and the outcome of the waits
        // becomes uniform over the CTA
        if (__syncthreads_or(!ok)) {
            dead = true;
            if (tid == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
        if (tid == 0 && jj + NST < njob) issue(j0 + jj + NST, stg);
    }
    if (dead) {  // uniform over the CTA
        // let copies still in flight land before the buffers are reused
        // (bounded); the block is finished with whatever it holds (the error
        // word is set)
        if (tid == 0)
            for (int q = 0; q < NST && q < njob; q++) (void)dev::mbar_wait(&bar[q], uses[q] & 1u, a.timeout_ns / 8);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NST; q++) uses[q] += static_cast<uint32_t>((njob - q + NST - 1) / NST);
    if constexpr (TCU) {
        // fragments -> element order (shared memory) -> the thread's own elements
        mma_store<D, GEN, PK, NS>(cfr, reinterpret_cast<QF*>(red));
#pragma unroll
        for (int s = 0; s < NACC; s++)
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                if ((TD % kThreads) == 0 || e < TD) acc[s][q] = red[s * TD + e];
            }
    }

    // ---- partial sums -> shared memory (the generalized form's Horner chain
    // mixes elements; a cluster reduces through it), cluster reduction into rank 0
    if (CHAIN || csize > 1) {
#pragma unroll
        for (int s = 0; s < NACC; s++)
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                if ((TD % kThreads) == 0 || e < TD) red[s * TD + e] = acc[s][q];
            }
    }
    if (csize > 1) {
        dev::cluster_sync();
        if (rank == 0) {
            for (int r = 1; r < csize; r++) {
#pragma unroll
                for (int s = 0; s < NACC; s++)
#pragma unroll
                    for (int q = 0; q < EPT; q++) {
                        const int e = tid + q * kThreads;
                        if ((TD % kThreads) == 0 || e < TD) acc[s][q] += dev::ld_dsmem(&red[s * TD + e], r);
                    }
            }
#pragma unroll
            for (int s = 0; s < NACC; s++)
#pragma unroll
                for (int q = 0; q < EPT; q++) {
                    const int e = tid + q * kThreads;
                    if ((TD % kThreads) == 0 || e < TD) red[s * TD + e] = acc[s][q];
                }
        }
        dev::cluster_sync();
        if (rank != 0) return !dead;
    }

    // ---- base case, the rest: right-hand side minus the block updates, then
    // back-substitution over the coupled groups in anti-diagonal order
    if constexpr (TT) {
        __syncthreads();
        // two-term form: the level sums of the Q chain through the diagonal
        // blocks of the chain factors (levels d-2 .. 1), then the mode-1
        // level: off(T) = c x Q_1 + (the A_1 sums already in the last slot)
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            __syncthreads();
            const int st = ipow(TE, l);
            const T* Pn = red + C::slotP(l + 1) * TD;
            T vp[EPT];
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                vp[q] = T(0);
                if ((TD % kThreads) != 0 && e >= TD) continue;
                const int i = (e / st) % TE, base = e - i * st;
                T p = red[C::slotP(l) * TD + e];
                for (int k = 0; k < TE; k++) p = dev::fmadd(Es[l * TC + i + TE * k], Pn[base + k * st], p);
                vp[q] = p;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                if ((TD % kThreads) != 0 && e >= TD) continue;
                red[C::slotP(l) * TD + e] = vp[q];
            }
        }
        __syncthreads();
        {
            const T* Pn = red + C::slotP(1) * TD;
            for (int e = tid; e < TD; e += kThreads) {
                const int i = e % TE, base = e - i;
                T off = red[(NACC - 1) * TD + e];
                for (int k = 0; k < TE; k++) off = dev::fmadd(Es[i + TE * k], Pn[base + k], off);
                Rs[e] -= off;
            }
        }
        __syncthreads();
    } else if constexpr (GEN) {
        __syncthreads();
        // Horner chain over the diagonal blocks (levels d-2 .. 1), then the
        // mode-1 level: off(T) = A(X with block T set to zero) restricted to T.
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            __syncthreads();
            const int st = ipow(TE, l);
            const T* Pn = red + C::slotP(l + 1) * TD;
            const T* Gn = red + C::slotG(l + 1) * TD;
            T vp[EPT], vg[EPT];
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                vp[q] = T(0); vg[q] = T(0);
                if ((TD % kThreads) != 0 && e >= TD) continue;
                const int i = (e / st) % TE, base = e - i * st;
                T p = red[C::slotP(l) * TD + e], g = red[C::slotG(l) * TD + e];
                for (int k = 0; k < TE; k++) {
                    const T ev = Es[l * TC + i + TE * k], dv = Ds[l * TC + i + TE * k];
                    const T pv = Pn[base + k * st], gv = Gn[base + k * st];
                    p = dev::fmadd(ev, pv, p);
                    g = dev::fmadd(ev, gv, dev::fmadd(dv, pv, g));
                }
                vp[q] = p; vg[q] = g;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = tid + q * kThreads;
                if ((TD % kThreads) != 0 && e >= TD) continue;
                red[C::slotP(l) * TD + e] = vp[q];
                red[C::slotG(l) * TD + e] = vg[q];
            }
        }
        __syncthreads();
        {
            const T* Pn = red + C::slotP(1) * TD;
            const T* Gn = red + C::slotG(1) * TD;
            for (int e = tid; e < TD; e += kThreads) {
                const int i = e % TE, base = e - i;
                T off = red[(NACC - 1) * TD + e];
                for (int k = 0; k < TE; k++) off = dev::fmadd(Es[i + TE * k], Gn[base + k], dev::fmadd(Ds[i + TE * k], Pn[base + k], off));
                Rs[e] -= off;
            }
        }
        __syncthreads();
    } else {
        // the thread's own elements (it loaded their right-hand side)
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int e = tid + q * kThreads;
            if ((TD % kThreads) == 0 || e < TD) Rs[e] -= acc[0][q];
        }
    }
    if constexpr (TT) {
        // park the level sums of the Q chain in the output blocks
#pragma unroll
        for (int l = 1; l < D; l++) {
            T* Pg = static_cast<T*>(a.P[l]) + t * TD;
            for (int e = tid; e < TD; e += kThreads) Pg[e] = red[C::slotP(l) * TD + e];
        }
        __syncthreads();
    }
    if constexpr (GEN) {
        // park the level sums of the block updates in the output blocks (the
        // in-block parts are added at the end), freeing `red` for Lin
#pragma unroll
        for (int l = 1; l < D; l++) {
            T* Pg = static_cast<T*>(a.P[l]) + t * TD;
            T* Gg = static_cast<T*>(a.G[l]) + t * TD;
            for (int e = tid; e < TD; e += kThreads) {
                Pg[e] = red[C::slotP(l) * TD + e];
                Gg[e] = red[C::slotG(l) * TD + e];
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < NACC * TD; e += kThreads) Lin[e] = T(0);
    if (CHAIN && C::PIN_IN_RING)  // the ring is free now: every copy has landed and been read
        for (int e = tid; e < C::NL * TD; e += kThreads) { Pin[e] = T(0); Gin[e] = T(0); }

    TileSmem<T, D, GENF> sm{Ds, Es, Rs, Rd, Xs, Pin, Gin, Lin, gs, gl, ng, bs, gidx};
    if constexpr (!C::INV_EARLY && !C::CPLX)
        for (int i = tid; i < ncg; i += kThreads)
            if (cg_moff[i] >= 0) status |= group_inverse<T, D, GENF>(sm, cg_list[i] & 0xfff, Minv + cg_moff[i]);
    __syncthreads();
    // all warps take part (a one-warp variant with warp barriers between the
    // anti-diagonals measured slower for FP32 too: the line sums of one step
    // are then serialised over fewer lanes)
    constexpr bool SOLO = false;
    if (!SOLO || tid < 32) {
        const int lane = tid & 31;
        for (int step = nsum - D; step >= 0; step--) {
            // elements of this anti-diagonal: line sums from the solved positions,
            // then the 1x1 groups are solved by their threads; members of coupled
            // groups publish their sums for the solving warp
            const int a0 = act_off[step], an = act_cnt[step];
            auto line_step = [&](int i, bool on) {
                const int code = act_list[a0 + i];
                const int e = ElemCode<D>::elem(code);
                int u[D], k0s[D], rem = e;
#pragma unroll
                for (int mu = 0; mu < D; mu++) {
                    u[mu] = rem % TE;
                    rem /= TE;
                    k0s[mu] = ElemCode<D>::k0(code, mu);
                }
                T L[NACC];
                pull_lines<T, D, GENF>(sm, e, u, k0s, L, on);
                if (!on) return;
                if (!ElemCode<D>::coupled(code)) {
                    status |= solve_single<T, D, GENF>(sm, e, u, L);
                } else {
#pragma unroll
                    for (int k = 0; k < NACC; k++) Lin[k * TD + e] = L[k];
                }
            };
            if constexpr (C::WARP_TERMS) {
                // whole warps take part (the line sums' term range is the warp's)
                for (int i0 = SOLO ? 0 : (tid & ~31); i0 < an; i0 += SOLO ? 32 : kThreads)
                    line_step(i0 + lane < an ? i0 + lane : i0, i0 + lane < an);
            } else {
                for (int i = SOLO ? lane : tid; i < an; i += SOLO ? 32 : kThreads) line_step(i, true);
            }
            const int c0 = cg_off[step], cn = cg_cnt[step];
            if (cn > 0) {
                if constexpr (SOLO) __syncwarp(); else __syncthreads();
                const int warp = SOLO ? 0 : tid >> 5, nw = SOLO ? 1 : kThreads >> 5;
                if constexpr (!C::CPLX) {  // no coupled groups with complex triangular coefficients
                    // groups of each class in this anti-diagonal (the list is
                    // ordered by class), then the warp tasks: up to 32 >> c
                    // groups of class c each
                    int cc[D];
#pragma unroll
                    for (int c = 0; c < D; c++) cc[c] = 0;
                    for (int i0 = 0; i0 < cn; i0 += 32) {
                        const int i = i0 + (tid & 31);
                        const int cls = i < cn ? cg_list[c0 + i] >> 12 : 0;
#pragma unroll
                        for (int c = 0; c < D; c++) cc[c] += __popc(__ballot_sync(0xffffffffu, cls == c + 1));
                    }
                    int ntask = 0;
#pragma unroll
                    for (int c = 1; c <= D; c++) ntask += (cc[c - 1] + (32 >> c) - 1) >> (5 - c);
                    for (int tk = warp; tk < ntask; tk += nw) {
                        int c = 1, first = 0, rest = tk;
                        for (; c < D; c++) {
                            const int nt = (cc[c - 1] + (32 >> c) - 1) >> (5 - c);
                            if (rest < nt) break;
                            rest -= nt;
                            first += cc[c - 1];
                        }
                        first += rest << (5 - c);
                        const int count = min(32 >> c, cc[c - 1] - (rest << (5 - c)));
                        status |= warp_group<T, D, GENF>(sm, c, cg_list + c0 + first, cg_moff + c0 + first, count, Minv);
                    }
                }
            }
            if constexpr (SOLO) __syncwarp(); else __syncthreads();
        }
    }
    if constexpr (SOLO) __syncthreads();
    if (status) atomicOr(a.err, status);

    // ---- write the solved block (and its intermediates)
    for (int e = tid; e < TD; e += kThreads) Xg[e] = Xs[e];
    if constexpr (TT) {
#pragma unroll
        for (int l = 1; l < D; l++) {
            T* Pg = static_cast<T*>(a.P[l]) + t * TD;
            for (int e = tid; e < TD; e += kThreads) Pg[e] += Pin[(l - 1) * TD + e];  // parked by this thread
        }
    }
    if constexpr (GEN) {
#pragma unroll
        for (int l = 1; l < D; l++) {
            T* Pg = static_cast<T*>(a.P[l]) + t * TD;
            T* Gg = static_cast<T*>(a.G[l]) + t * TD;
            for (int e = tid; e < TD; e += kThreads) {  // the same thread parked Pg[e], Gg[e]
                Pg[e] += Pin[(l - 1) * TD + e];
                Gg[e] += Gin[(l - 1) * TD + e];
            }
        }
    }
    return !dead;
}

// Compiled for the same resident count as the persistent kernel, so that a
// block runs the same machine code (the same contractions into FMAs) in both
// schedules.
template <typename T, int D, int GENF>
__global__ void __launch_bounds__(kThreads, WaveCfg<T, D, GENF>::MINB) k_wave(const WaveArgs a) {
    using C = WaveCfg<T, D, GENF>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::oBar);
    const int csize = a.csize;
    const int rank = csize > 1 ? static_cast<int>(dev::cluster_rank()) : 0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < C::NST; q++) dev::mbar_init(&bar[q], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses[C::NST] = {};
    (void)wave_tile<T, D, GENF>(a, a.tiles[blockIdx.x / csize], rank, csize, uses, bar);
}

template <typename T, int D, int GEN>
cudaError_t prepare_wave_t() {
    using C = WaveCfg<T, D, GEN>;
    return cudaFuncSetAttribute(k_wave<T, D, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::smem));
}

template <typename T, int D, int GEN>
cudaError_t launch_wave_t(const WaveArgs& a, cudaStream_t s) {
    using C = WaveCfg<T, D, GEN>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(a.ntiles) * static_cast<unsigned>(a.csize), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = C::smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (a.csize > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = static_cast<unsigned>(a.csize);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, k_wave<T, D, GEN>, a);
}

}  // namespace tsylv
