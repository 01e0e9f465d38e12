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
#include "tsylv_internal.h"

namespace tsylv {

template <typename T, int D, bool GENF>
struct WaveCfg {
    static constexpr int TE = tile_extent(D);
    static constexpr int TD = ipow(TE, D);
    static constexpr int TC = TE * TE;
    static constexpr int EPT = (TD + kThreads - 1) / kThreads;
    static constexpr bool GEN = GENF && D >= 2;
    static constexpr int NACC = GEN ? 2 * (D - 1) + 1 : 1;
    static constexpr int NL = GEN ? D - 1 : 0;  // stored levels l = 1..d-1
    static constexpr int STAGE = 2 * TD + 2 * TC;
    static constexpr int oStage = 0;
    static constexpr int oRed = 2 * STAGE;
    static constexpr int oR = oRed + NACC * TD;
    static constexpr int oX = oR + TD;
    static constexpr int oPin = oX + TD;
    static constexpr int oGin = oPin + NL * TD;
    static constexpr int oD = oGin + NL * TD;
    static constexpr int oE = oD + D * TC;
    static constexpr int oEnd = oE + (GEN ? D * TC : 0);
    static constexpr size_t oBar = ((oEnd * sizeof(T)) + 15) / 16 * 16;
    static constexpr size_t oMeta = oBar + 16;
    static constexpr size_t smem = oMeta + (2 * D * TE + 3 * D + 4) * sizeof(int);
    static constexpr int slotP(int l) { return 2 * (D - 1 - l); }
    static constexpr int slotG(int l) { return 2 * (D - 1 - l) + 1; }
};

// acc[q] += (S x_MU M)[e_q] for the thread's elements e_q = tid + q*kThreads:
//   y(.., i, ..) = sum_k M(i, k) S(.., k, ..),  M a TE x TE column-major tile.
template <typename T, int D, int MU, int EPT>
__device__ __forceinline__ void prod_acc(T (&acc)[EPT], const T* __restrict__ M, const T* __restrict__ S) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = (e / st) % TE;
        const int base = e - i * st;
        T s = acc[q];
#pragma unroll
        for (int k = 0; k < TE; k++) s = dev::fmadd(M[i + TE * k], S[base + k * st], s);
        acc[q] = s;
    }
}

// acc[q] += (S1 x_MU M1 + S2 x_MU M2)[e_q]
template <typename T, int D, int MU, int EPT>
__device__ __forceinline__ void prod_acc2(T (&acc)[EPT], const T* __restrict__ M1, const T* __restrict__ S1,
                                          const T* __restrict__ M2, const T* __restrict__ S2) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = (e / st) % TE;
        const int base = e - i * st;
        T s = acc[q];
#pragma unroll
        for (int k = 0; k < TE; k++) {
            s = dev::fmadd(M1[i + TE * k], S1[base + k * st], s);
            s = dev::fmadd(M2[i + TE * k], S2[base + k * st], s);
        }
        acc[q] = s;
    }
}

// Compile-time dispatch of one block-update job of level L.
template <typename T, int D, bool GEN, int L>
struct JobCompute {
    template <int NACC, int EPT>
    __device__ __forceinline__ static void run(T (&acc)[NACC][EPT], const T* stage) {
        constexpr int TE = tile_extent(D);
        constexpr int TD = ipow(TE, D);
        constexpr int TC = TE * TE;
        const T* S1 = stage;
        const T* S2 = stage + TD;
        const T* M1 = stage + 2 * TD;
        const T* M2 = stage + 2 * TD + TC;
        if constexpr (!GEN) {
            prod_acc<T, D, L, EPT>(acc[0], M1, S1);  // Laplace: level L = mode L
        } else {
            constexpr int MU = D - 1 - L;            // modes d-1, ..., 0
            if constexpr (L == 0) {
                // L^P_{d-1} += X x C,  L^G_{d-1} += X x A
                prod_acc<T, D, MU, EPT>(acc[0], M1, S1);
                prod_acc<T, D, MU, EPT>(acc[1], M2, S1);
            } else if constexpr (MU >= 1) {
                // L^P_mu += P_{mu+1} x C,  L^G_mu += G_{mu+1} x C + P_{mu+1} x A
                prod_acc<T, D, MU, EPT>(acc[2 * L], M1, S1);
                prod_acc2<T, D, MU, EPT>(acc[2 * L + 1], M1, S2, M2, S1);
            } else {
                // L_0 += G_1 x C_0 + P_1 x A_0
                prod_acc2<T, D, 0, EPT>(acc[NACC - 1], M1, S2, M2, S1);
            }
        }
    }
};

template <typename T, int D, bool GEN, int L = 0>
__device__ __forceinline__ void dispatch_job(int level, T (&acc)[WaveCfg<T, D, GEN>::NACC][WaveCfg<T, D, GEN>::EPT],
                                             const T* stage) {
    if constexpr (L < D) {
        if (level == L)
            JobCompute<T, D, WaveCfg<T, D, GEN>::GEN, L>::run(acc, stage);
        else
            dispatch_job<T, D, GEN, L + 1>(level, acc, stage);
    }
}

// Dense Gaussian elimination with partial pivoting for one coupled group
// (s <= 2^d unknowns).  Returns false for a pivot below 16 eps max|M|.
template <typename T, int SMAX>
__device__ bool group_gepp(int s, T* M, T* r) {
    T big = 0;
    for (int i = 0; i < s * s; i++) big = fmax(big, fabs(M[i]));
    const T tiny = T(16) * dev::Eps<T>::v * big;
    for (int c = 0; c < s; c++) {
        int p = c;
        T best = fabs(M[c * SMAX + c]);
        for (int q = c + 1; q < s; q++) {
            T v = fabs(M[q * SMAX + c]);
            if (v > best) { best = v; p = q; }
        }
        if (!(best > tiny)) return false;
        if (p != c) {
            for (int k = 0; k < s; k++) { T t = M[c * SMAX + k]; M[c * SMAX + k] = M[p * SMAX + k]; M[p * SMAX + k] = t; }
            T t = r[c]; r[c] = r[p]; r[p] = t;
        }
        for (int q = c + 1; q < s; q++) {
            T f = M[q * SMAX + c] / M[c * SMAX + c];
            for (int k = c; k < s; k++) M[q * SMAX + k] -= f * M[c * SMAX + k];
            r[q] -= f * r[c];
        }
    }
    for (int c = s - 1; c >= 0; c--) {
        T v = r[c];
        for (int k = c + 1; k < s; k++) v -= M[c * SMAX + k] * r[k];
        r[c] = v / M[c * SMAX + c];
    }
    return true;
}

template <typename T, int D, bool GEN>
struct TileSmem {
    const T* Ds;   // [D][TC] diagonal tiles of A
    const T* Es;   // [D][TC] diagonal tiles of C (generalized)
    const T* Rs;   // right-hand side of the diagonal-block equation
    T* Xs;         // solution (0 where not yet solved)
    T* Pin;        // [NL][TD] in-block intermediates (generalized)
    T* Gin;
    const int* gs; // [D][TE] group start
    const int* gl; // [D][TE] group length (1 or 2)
    const int* ng; // [D] groups per mode
    const int* bs; // [D] block extent
};

// Solve one coupled group g of the diagonal-block equation (element-level
// version of the block recurrence: partial sums beyond the group along each
// mode, the group system, then completion of the in-block intermediates).
template <typename T, int D, bool GEN>
__device__ int solve_group(const TileSmem<T, D, GEN>& sm, const int (&g)[D]) {
    constexpr int TE = tile_extent(D);
    constexpr int TD = ipow(TE, D);
    constexpr int TC = TE * TE;
    constexpr int SMAX = 1 << D;
    int a[D], s[D], smem_st[D], st[D];
    int S = 1, o = 0;
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        a[mu] = sm.gs[mu * TE + g[mu]];
        s[mu] = sm.gl[mu * TE + g[mu]];
        smem_st[mu] = S;
        S *= s[mu];
        st[mu] = ipow(TE, mu);
        o += a[mu] * st[mu];
    }
    auto Dm = [&](int mu, int i, int k) -> T { return sm.Ds[mu * TC + i + TE * k]; };
    auto Em = [&](int mu, int i, int k) -> T { return sm.Es[mu * TC + i + TE * k]; };
    int status = 0;
    if (S == 1) {
        // ------------------------------------------------ single unknown
        T x;
        T mag = 0;
        T diag = 0;
        if constexpr (!GEN) {
            T r = sm.Rs[o];
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                const T dd = Dm(mu, a[mu], a[mu]);
                diag += dd;
                mag += fabs(dd);
                for (int k = a[mu] + 1; k < sm.bs[mu]; k++) r -= Dm(mu, a[mu], k) * sm.Xs[o + (k - a[mu]) * st[mu]];
            }
            x = r / diag;
        } else {
            T p0[D], g0[D];
            {
                constexpr int mu = D - 1;
                T p = 0, q = 0;
                for (int k = a[mu] + 1; k < sm.bs[mu]; k++) {
                    const T xv = sm.Xs[o + (k - a[mu]) * st[mu]];
                    p += Em(mu, a[mu], k) * xv;
                    q += Dm(mu, a[mu], k) * xv;
                }
                p0[mu] = p;
                g0[mu] = q;
            }
#pragma unroll
            for (int l = D - 2; l >= 1; l--) {
                const T ep = Em(l, a[l], a[l]), dp = Dm(l, a[l], a[l]);
                T p = ep * p0[l + 1];
                T q = ep * g0[l + 1] + dp * p0[l + 1];
                const T* Pn = sm.Pin + (l + 1 - 1) * TD;
                const T* Gn = sm.Gin + (l + 1 - 1) * TD;
                for (int k = a[l] + 1; k < sm.bs[l]; k++) {
                    const int oo = o + (k - a[l]) * st[l];
                    p += Em(l, a[l], k) * Pn[oo];
                    q += Em(l, a[l], k) * Gn[oo] + Dm(l, a[l], k) * Pn[oo];
                }
                p0[l] = p;
                g0[l] = q;
            }
            T off = Em(0, a[0], a[0]) * g0[1] + Dm(0, a[0], a[0]) * p0[1];
            {
                const T* Pn = sm.Pin;
                const T* Gn = sm.Gin;
                for (int k = a[0] + 1; k < sm.bs[0]; k++) {
                    const int oo = o + (k - a[0]);
                    off += Em(0, a[0], k) * Gn[oo] + Dm(0, a[0], k) * Pn[oo];
                }
            }
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                T t = Dm(mu, a[mu], a[mu]);
#pragma unroll
                for (int eta = 0; eta < D; eta++)
                    if (eta != mu) t *= Em(eta, a[eta], a[eta]);
                diag += t;
                mag += fabs(t);
            }
            x = (sm.Rs[o] - off) / diag;
            // completion of the in-block intermediates at this position
            T pc = Em(D - 1, a[D - 1], a[D - 1]) * x;
            T gc = Dm(D - 1, a[D - 1], a[D - 1]) * x;
            sm.Pin[(D - 2) * TD + o] = p0[D - 1] + pc;
            sm.Gin[(D - 2) * TD + o] = g0[D - 1] + gc;
#pragma unroll
            for (int l = D - 2; l >= 1; l--) {
                const T ep = Em(l, a[l], a[l]), dp = Dm(l, a[l], a[l]);
                gc = ep * gc + dp * pc;
                pc = ep * pc;
                sm.Pin[(l - 1) * TD + o] = p0[l] + pc;
                sm.Gin[(l - 1) * TD + o] = g0[l] + gc;
            }
        }
        if (!(fabs(diag) > T(16) * dev::Eps<T>::v * mag)) status |= kErrSingular;
        if (!isfinite(x)) status |= kErrNonfinite;
        sm.Xs[o] = x;
        return status;
    }
    // ---------------------------------------------------- coupled group
    int om[SMAX];
    int um[SMAX][D];
    for (int m = 0; m < S; m++) {
        int oo = 0;
#pragma unroll
        for (int mu = 0; mu < D; mu++) {
            um[m][mu] = a[mu] + (m / smem_st[mu]) % s[mu];
            oo += um[m][mu] * st[mu];
        }
        om[m] = oo;
    }
    T r[SMAX];
    T M[SMAX * SMAX];
    T P0[D][SMAX], G0[D][SMAX];
    if constexpr (!GEN) {
        for (int m = 0; m < S; m++) {
            T v = sm.Rs[om[m]];
#pragma unroll
            for (int mu = 0; mu < D; mu++) {
                const int u = um[m][mu];
                for (int k = a[mu] + s[mu]; k < sm.bs[mu]; k++) v -= Dm(mu, u, k) * sm.Xs[om[m] + (k - u) * st[mu]];
            }
            r[m] = v;
            for (int m2 = 0; m2 < S; m2++) {
                T e = 0;
#pragma unroll
                for (int mu = 0; mu < D; mu++) {
                    bool same = true;
#pragma unroll
                    for (int eta = 0; eta < D; eta++)
                        if (eta != mu && um[m][eta] != um[m2][eta]) same = false;
                    if (same) e += Dm(mu, um[m][mu], um[m2][mu]);
                }
                M[m * SMAX + m2] = e;
            }
        }
    } else {
        for (int m = 0; m < S; m++) {
            constexpr int mu = D - 1;
            const int u = um[m][mu];
            T p = 0, q = 0;
            for (int k = a[mu] + s[mu]; k < sm.bs[mu]; k++) {
                const T xv = sm.Xs[om[m] + (k - u) * st[mu]];
                p += Em(mu, u, k) * xv;
                q += Dm(mu, u, k) * xv;
            }
            P0[mu][m] = p;
            G0[mu][m] = q;
        }
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            const T* Pn = sm.Pin + l * TD;  // level l + 1
            const T* Gn = sm.Gin + l * TD;
            for (int m = 0; m < S; m++) {
                const int u = um[m][l];
                T p = 0, q = 0;
                for (int k = a[l]; k < a[l] + s[l]; k++) {
                    const int m2 = m + (k - u) * smem_st[l];
                    p += Em(l, u, k) * P0[l + 1][m2];
                    q += Em(l, u, k) * G0[l + 1][m2] + Dm(l, u, k) * P0[l + 1][m2];
                }
                for (int k = a[l] + s[l]; k < sm.bs[l]; k++) {
                    const int oo = om[m] + (k - u) * st[l];
                    p += Em(l, u, k) * Pn[oo];
                    q += Em(l, u, k) * Gn[oo] + Dm(l, u, k) * Pn[oo];
                }
                P0[l][m] = p;
                G0[l][m] = q;
            }
        }
        for (int m = 0; m < S; m++) {
            const int u = um[m][0];
            T off = 0;
            for (int k = a[0]; k < a[0] + s[0]; k++) {
                const int m2 = m + (k - u) * smem_st[0];
                off += Em(0, u, k) * G0[1][m2] + Dm(0, u, k) * P0[1][m2];
            }
            for (int k = a[0] + s[0]; k < sm.bs[0]; k++) {
                const int oo = om[m] + (k - u);
                off += Em(0, u, k) * sm.Gin[oo] + Dm(0, u, k) * sm.Pin[oo];
            }
            r[m] = sm.Rs[om[m]] - off;
            for (int m2 = 0; m2 < S; m2++) {
                T e = 0;
#pragma unroll
                for (int mu = 0; mu < D; mu++) {
                    T t = Dm(mu, um[m][mu], um[m2][mu]);
#pragma unroll
                    for (int eta = 0; eta < D; eta++)
                        if (eta != mu) t *= Em(eta, um[m][eta], um[m2][eta]);
                    e += t;
                }
                M[m * SMAX + m2] = e;
            }
        }
    }
    if (!group_gepp<T, SMAX>(S, M, r)) status |= kErrSingular;
    for (int m = 0; m < S; m++) {
        if (!isfinite(r[m])) status |= kErrNonfinite;
        sm.Xs[om[m]] = r[m];
    }
    if constexpr (GEN) {
        T pc[D][SMAX], gc[D][SMAX];
        for (int m = 0; m < S; m++) {
            constexpr int mu = D - 1;
            const int u = um[m][mu];
            T p = 0, q = 0;
            for (int k = a[mu]; k < a[mu] + s[mu]; k++) {
                const int m2 = m + (k - u) * smem_st[mu];
                p += Em(mu, u, k) * r[m2];
                q += Dm(mu, u, k) * r[m2];
            }
            pc[mu][m] = p;
            gc[mu][m] = q;
        }
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            for (int m = 0; m < S; m++) {
                const int u = um[m][l];
                T p = 0, q = 0;
                for (int k = a[l]; k < a[l] + s[l]; k++) {
                    const int m2 = m + (k - u) * smem_st[l];
                    p += Em(l, u, k) * pc[l + 1][m2];
                    q += Em(l, u, k) * gc[l + 1][m2] + Dm(l, u, k) * pc[l + 1][m2];
                }
                pc[l][m] = p;
                gc[l][m] = q;
            }
        }
        for (int m = 0; m < S; m++) {
#pragma unroll
            for (int l = 1; l < D; l++) {
                sm.Pin[(l - 1) * TD + om[m]] = P0[l][m] + pc[l][m];
                sm.Gin[(l - 1) * TD + om[m]] = G0[l][m] + gc[l][m];
            }
        }
    }
    return status;
}

template <typename T, int D, bool GENF>
__global__ void __launch_bounds__(kThreads) k_wave(const WaveArgs a) {
    using C = WaveCfg<T, D, GENF>;
    constexpr int TE = C::TE, TD = C::TD, TC = C::TC, EPT = C::EPT, NACC = C::NACC;
    constexpr bool GEN = C::GEN;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* sbase = reinterpret_cast<T*>(smem_raw);
    T* stage = sbase + C::oStage;
    T* red = sbase + C::oRed;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::oBar);
    int* meta = reinterpret_cast<int*>(smem_raw + C::oMeta);
    int* gs = meta;                  // [D][TE]
    int* gl = gs + D * TE;           // [D][TE]
    int* ng = gl + D * TE;           // [D]
    int* bs = ng + D;                // [D]
    int* flag = bs + D;              // [4]

    const int tid = threadIdx.x;
    const int csize = a.csize;
    const int rank = csize > 1 ? static_cast<int>(dev::cluster_rank()) : 0;
    const int tix = blockIdx.x / csize;
    const long long t = a.tiles[tix];
    int I[D];
#pragma unroll
    for (int mu = 0; mu < D; mu++) I[mu] = static_cast<int>((t / a.tstride[mu]) % a.nb[mu]);

    // ---- job list: level L covers mode L (Laplace) or d-1-L (generalized)
    int cnt[D], w[D];
    long long W = 0;
#pragma unroll
    for (int L = 0; L < D; L++) {
        const int mu = GEN ? D - 1 - L : L;
        cnt[L] = a.hi[mu] - 1 - I[mu];
        if (cnt[L] < 0) cnt[L] = 0;
        w[L] = GEN ? ((L == 0 || L == D - 1) ? 2 : 3) : 1;
        W += static_cast<long long>(cnt[L]) * w[L];
    }
    const long long wlo = W * rank / csize, whi = W * (rank + 1) / csize;
    int j0 = 0, j1 = 0, jt = 0;
    {
        long long cw = 0;
        bool f0 = false, f1 = false;
        for (int L = 0; L < D; L++) {
            for (int k = 0; k < cnt[L]; k++) {
                if (!f0 && cw >= wlo) { j0 = jt; f0 = true; }
                if (!f1 && cw >= whi) { j1 = jt; f1 = true; }
                cw += w[L];
                jt++;
            }
        }
        if (!f0) j0 = jt;
        if (!f1) j1 = jt;
    }
    const int njob = j1 - j0;

    // job j -> (level, source block J')
    auto decode = [&](int j, int& L, int& Jp) {
        L = 0;
        while (L < D - 1 && j >= cnt[L]) { j -= cnt[L]; L++; }
        const int mu = GEN ? D - 1 - L : L;
        Jp = I[mu] + 1 + j;
    };
    auto issue = [&](int j, int stg) {
        int L, Jp;
        decode(j, L, Jp);
        const int mu = GEN ? D - 1 - L : L;
        const long long ts = t + static_cast<long long>(Jp - I[mu]) * a.tstride[mu];
        const long long tri = static_cast<long long>(Jp) * (Jp + 1) / 2 + I[mu];
        T* sb = stage + stg * C::STAGE;
        const T* S1;
        const T* S2 = nullptr;
        const T* M1;
        const T* M2 = nullptr;
        if (!GEN) {
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

    if (tid == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
        flag[0] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        if (njob > 0) issue(j0, 0);
        if (njob > 1) issue(j0 + 1, 1);
    }
    bool dead = false;
    for (int jj = 0; jj < njob && !dead; jj++) {
        const int stg = jj & 1;
        const bool ok = dev::mbar_wait(&bar[stg], static_cast<uint32_t>((jj >> 1) & 1), a.timeout_ns);
        if (__syncthreads_or(!ok)) {
            dead = true;
            if (tid == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
        int L, Jp;
        decode(j0 + jj, L, Jp);
        dispatch_job<T, D, GENF>(L, acc, stage + stg * C::STAGE);
        __syncthreads();
        if (tid == 0 && jj + 2 < njob) {
            dev::fence_proxy_async();
            issue(j0 + jj + 2, stg);
        }
    }
    if (dead && tid == 0) {
        // let copies still in flight land before the buffers go away (bounded)
        for (int jj = 0; jj < 2 && jj < njob; jj++) (void)dev::mbar_wait(&bar[jj], 0, a.timeout_ns / 8);
    }

    // ---- partial sums -> shared memory, cluster reduction into rank 0
#pragma unroll
    for (int s = 0; s < NACC; s++)
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int e = tid + q * kThreads;
            if ((TD % kThreads) == 0 || e < TD) red[s * TD + e] = acc[s][q];
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
        if (rank != 0) return;
    }

    // ---- rank 0: base case of block T
    T* Rs = sbase + C::oR;
    T* Xs = sbase + C::oX;
    T* Pin = sbase + C::oPin;
    T* Gin = sbase + C::oGin;
    T* Ds = sbase + C::oD;
    T* Es = sbase + C::oE;
    T* Xg = static_cast<T*>(a.X) + t * TD;
    for (int idx = tid; idx < D * TC; idx += kThreads) {
        const int mu = idx / TC, e = idx % TC;
        const long long tri = static_cast<long long>(I[mu]) * (I[mu] + 1) / 2 + I[mu];
        Ds[idx] = static_cast<const T*>(a.At[mu])[tri * TC + e];
        if (GEN) Es[idx] = static_cast<const T*>(a.Ct[mu])[tri * TC + e];
    }
    for (int e = tid; e < TD; e += kThreads) {
        Rs[e] = Xg[e];
        Xs[e] = T(0);
    }
    if (GEN)
        for (int e = tid; e < C::NL * TD; e += kThreads) { Pin[e] = T(0); Gin[e] = T(0); }
    if (tid < D) bs[tid] = a.bsize[tid][I[tid]];
    __syncthreads();
    if (tid < D) {
        const int mu = tid, b = bs[mu];
        int n = 0, i = 0;
        while (i < b) {
            if (i + 1 < b && Ds[mu * TC + (i + 1) + TE * i] != T(0)) {
                gs[mu * TE + n] = i; gl[mu * TE + n] = 2; i += 2;
            } else {
                gs[mu * TE + n] = i; gl[mu * TE + n] = 1; i += 1;
            }
            n++;
        }
        ng[mu] = n;
    }
    if constexpr (GEN) {
        // Horner chain over the diagonal blocks (levels d-2 .. 1), then the
        // mode-1 level: off(T) = A(X with block T set to zero) restricted to T.
#pragma unroll
        for (int l = D - 2; l >= 1; l--) {
            __syncthreads();
            constexpr int dummy = 0;
            (void)dummy;
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
                    p += ev * pv;
                    g += ev * gv + dv * pv;
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
                for (int k = 0; k < TE; k++) off += Es[i + TE * k] * Gn[base + k] + Ds[i + TE * k] * Pn[base + k];
                Rs[e] -= off;
            }
        }
    } else {
        for (int e = tid; e < TD; e += kThreads) Rs[e] -= red[e];
    }
    __syncthreads();

    // ---- back-substitution over coupled groups, anti-diagonal order
    TileSmem<T, D, GEN> sm{Ds, Es, Rs, Xs, Pin, Gin, gs, gl, ng, bs};
    int nsum = 0, nthr = 1;
#pragma unroll
    for (int mu = 0; mu < D; mu++) nsum += ng[mu];
#pragma unroll
    for (int mu = 1; mu < D; mu++) nthr *= ng[mu];
    int status = 0;
    for (int step = nsum - D; step >= 0; step--) {
        for (int j = tid; j < nthr; j += kThreads) {
            int g[D];
            int rem = j, sum = 0;
#pragma unroll
            for (int mu = 1; mu < D; mu++) { g[mu] = rem % ng[mu]; rem /= ng[mu]; sum += g[mu]; }
            g[0] = step - sum;
            if (g[0] >= 0 && g[0] < ng[0]) status |= solve_group<T, D, GEN>(sm, g);
        }
        __syncthreads();
    }
    if (status) atomicOr(a.err, status);

    // ---- write the solved block (and its intermediates)
    for (int e = tid; e < TD; e += kThreads) Xg[e] = Xs[e];
    if constexpr (GEN) {
#pragma unroll
        for (int l = 1; l < D; l++) {
            T* Pg = static_cast<T*>(a.P[l]) + t * TD;
            T* Gg = static_cast<T*>(a.G[l]) + t * TD;
            for (int e = tid; e < TD; e += kThreads) {
                Pg[e] = red[C::slotP(l) * TD + e] + Pin[(l - 1) * TD + e];
                Gg[e] = red[C::slotG(l) * TD + e] + Gin[(l - 1) * TD + e];
            }
        }
    }
}

template <typename T, int D, bool GEN>
cudaError_t prepare_wave_t() {
    using C = WaveCfg<T, D, GEN>;
    return cudaFuncSetAttribute(k_wave<T, D, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::smem));
}

template <typename T, int D, bool GEN>
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

template <typename T>
cudaError_t prepare_wave_impl() {
    cudaError_t e = cudaSuccess;
    if ((e = prepare_wave_t<T, 1, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 2, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 2, true>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 3, false>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 3, true>()) != cudaSuccess) return e;
    if ((e = prepare_wave_t<T, 4, false>()) != cudaSuccess) return e;
    return prepare_wave_t<T, 4, true>();
}

template <typename T>
cudaError_t launch_wave_impl(int d, bool gen, const WaveArgs& a, cudaStream_t s) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2: return launch_wave_t<T, 1, false>(a, s);
        case 3: return launch_wave_t<T, 1, false>(a, s);  // d = 1: both forms coincide
        case 4: return launch_wave_t<T, 2, false>(a, s);
        case 5: return launch_wave_t<T, 2, true>(a, s);
        case 6: return launch_wave_t<T, 3, false>(a, s);
        case 7: return launch_wave_t<T, 3, true>(a, s);
        case 8: return launch_wave_t<T, 4, false>(a, s);
        case 9: return launch_wave_t<T, 4, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tsylv
