// Operator application on the block tensor, one block per call: the per-block
// function of the residual kernels (FP64, DF64 = float pairs on the FP32 pipes,
// FP32), shared by the stand-alone apply launches and by the fused
// solve + residual step of the refinement.
#pragma once

#include "apply_kernel.cuh"
#include "device_common.cuh"

namespace tsylv {
namespace apply_detail {

// DF64 helpers: (h, l) unevaluated pairs of floats.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (sh, sl) += (ah + al) * (xh + xl), dropping al * xl
__device__ __forceinline__ void df_fma(float ah, float al, float xh, float xl, float& sh, float& sl) {
    const float p = __fmul_rn(ah, xh);  // rounded product, never fused into the sum below
    const float e = fmaf(ah, xh, -p);    // exact: ah * xh = p + e
    const float t = fmaf(ah, xl, fmaf(al, xh, e));
    float s, err;
    two_sum(sh, p, s, err);
    sh = s;
    sl += err + t;
}
__device__ __forceinline__ void df_norm(float h, float l, float& oh, float& ol) {
    oh = h + l;
    ol = l - (oh - h);
}
__device__ __forceinline__ double df_to_double(float h, float l) { return static_cast<double>(h) + static_cast<double>(l); }

}  // namespace apply_detail
}  // namespace tsylv

namespace tsylv {
namespace apply_detail {

template <int D, int M>
struct ApplyCfg {
    static constexpr int TE = tile_extent(D);
    static constexpr int TD = ipow(TE, D);
    static constexpr int TC = TE * TE;
    static constexpr int EPT = (TD + kThreads - 1) / kThreads;
    // one stage: S1, S2 (P x TD each), M1, M2 (P x TC each), in 8-byte units
    static constexpr int STAGE_BYTES = (2 * TD + 2 * TC) * 8;
    // stages of the bulk-copy ring (every block is independent here: the
    // ring only has to cover the copy latency)
    static constexpr int NST = 4;
    static constexpr size_t oBar = NST * STAGE_BYTES;
    static constexpr size_t oRed = oBar + 8 * NST;
    static constexpr size_t smem = oRed + 2 * (kThreads / 32) * sizeof(double);
};

// y[q] += (M x_MU S)[e_q]: FP64
template <int D, int MU, int EPT>
__device__ __forceinline__ void acc_f64(double (&y)[EPT], const double* __restrict__ M, const double* __restrict__ S) {
    constexpr int TE = tile_extent(D), TD = ipow(TE, D), st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = row_of<TE, st>(e), base = e - i * st;
        double s = y[q];
#pragma unroll
        for (int k = 0; k < TE; k++) s = fma(M[i + TE * k], S[base + k * st], s);
        y[q] = s;
    }
}

// (yh, yl)[q] += (M x_MU S)[e_q]: DF64, M and S given as (hi, lo) float tiles
template <int D, int MU, int EPT>
__device__ __forceinline__ void acc_df(float (&yh)[EPT], float (&yl)[EPT], const float* __restrict__ Mh,
                                       const float* __restrict__ Ml, const float* __restrict__ Sh,
                                       const float* __restrict__ Sl) {
    constexpr int TE = tile_extent(D), TD = ipow(TE, D), st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = row_of<TE, st>(e), base = e - i * st;
        float h = yh[q], l = yl[q];
#pragma unroll
        for (int k = 0; k < TE; k++) df_fma(Mh[i + TE * k], Ml[i + TE * k], Sh[base + k * st], Sl[base + k * st], h, l);
        yh[q] = h;
        yl[q] = l;
    }
}

// (yh, yl)[q] += (M x_MU S)[e_q]: DF64, M a (hi, lo) float tile, S an exact float tile
template <int D, int MU, int EPT>
__device__ __forceinline__ void acc_dfh(float (&yh)[EPT], float (&yl)[EPT], const float* __restrict__ Mh,
                                        const float* __restrict__ Ml, const float* __restrict__ Sh) {
    constexpr int TE = tile_extent(D), TD = ipow(TE, D), st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = row_of<TE, st>(e), base = e - i * st;
        float h = yh[q], l = yl[q];
#pragma unroll
        for (int k = 0; k < TE; k++) {
            const float mh = Mh[i + TE * k], ml = Ml[i + TE * k], x = Sh[base + k * st];
            const float pr = __fmul_rn(mh, x);  // rounded product, never fused into the sum below
            const float t = fmaf(ml, x, fmaf(mh, x, -pr));  // exact low part of mh x, plus ml x
            float sum, err;
            two_sum(h, pr, sum, err);
            h = sum;
            l += err + t;
        }
        yh[q] = h;
        yl[q] = l;
    }
}

// y[q] += (M x_MU S)[e_q]: FP32
template <int D, int MU, int EPT>
__device__ __forceinline__ void acc_f32(float (&y)[EPT], const float* __restrict__ M, const float* __restrict__ S) {
    constexpr int TE = tile_extent(D), TD = ipow(TE, D), st = ipow(TE, MU);
#pragma unroll
    for (int q = 0; q < EPT; q++) {
        const int e = threadIdx.x + q * kThreads;
        if ((TD % kThreads) != 0 && e >= TD) continue;
        const int i = row_of<TE, st>(e), base = e - i * st;
        float v = y[q];
#pragma unroll
        for (int k = 0; k < TE; k++) v = fmaf(M[i + TE * k], S[base + k * st], v);
        y[q] = v;
    }
}

template <int D, int MD, int MU>
__device__ __forceinline__ void do_job(int kind, const unsigned char* stg, double (&y1)[ApplyCfg<D, MD>::EPT],
                                       double (&y2)[ApplyCfg<D, MD>::EPT], float (&h1)[ApplyCfg<D, MD>::EPT],
                                       float (&l1)[ApplyCfg<D, MD>::EPT], float (&h2)[ApplyCfg<D, MD>::EPT],
                                       float (&l2)[ApplyCfg<D, MD>::EPT]) {
    using C = ApplyCfg<D, MD>;
    constexpr int TD = C::TD, TC = C::TC, EPT = C::EPT;
    if constexpr (MD == kModeF32) {
        // same staging layout as DF64, the low words unused
        const float* S1 = reinterpret_cast<const float*>(stg);
        const float* S2 = S1 + 2 * TD;
        const float* M1 = S1 + 4 * TD;
        const float* M2 = M1 + 2 * TC;
        if (kind == kApplyLaplace) {
            acc_f32<D, MU, EPT>(h1, M1, S1);
        } else if (kind == kApplyFirst) {
            acc_f32<D, MU, EPT>(h1, M1, S1);
            acc_f32<D, MU, EPT>(h2, M2, S1);
        } else if (kind == kApplyMiddle) {
            acc_f32<D, MU, EPT>(h1, M1, S1);
            acc_f32<D, MU, EPT>(h2, M1, S2);
            acc_f32<D, MU, EPT>(h2, M2, S1);
        } else {
            acc_f32<D, MU, EPT>(h1, M1, S2);
            acc_f32<D, MU, EPT>(h1, M2, S1);
        }
    } else if constexpr (MD == kModeF64) {
        const double* S1 = reinterpret_cast<const double*>(stg);
        const double* S2 = S1 + TD;
        const double* M1 = S2 + TD;
        const double* M2 = M1 + TC;
        if (kind == kApplyLaplace) {
            acc_f64<D, MU, EPT>(y1, M1, S1);
        } else if (kind == kApplyFirst) {
            acc_f64<D, MU, EPT>(y1, M1, S1);
            acc_f64<D, MU, EPT>(y2, M2, S1);
        } else if (kind == kApplyMiddle) {
            acc_f64<D, MU, EPT>(y1, M1, S1);
            acc_f64<D, MU, EPT>(y2, M1, S2);
            acc_f64<D, MU, EPT>(y2, M2, S1);
        } else {
            acc_f64<D, MU, EPT>(y1, M1, S2);
            acc_f64<D, MU, EPT>(y1, M2, S1);
        }
    } else if constexpr (MD == kModeDFh) {
        // same staging layout as DF64 (the source's low words not copied);
        // only the kinds with one source occur
        const float* S1h = reinterpret_cast<const float*>(stg);
        const float* M1h = S1h + 4 * TD;
        const float* M1l = M1h + TC;
        const float* M2h = M1l + TC;
        const float* M2l = M2h + TC;
        if (kind == kApplyLaplace) {
            acc_dfh<D, MU, EPT>(h1, l1, M1h, M1l, S1h);
        } else {
            acc_dfh<D, MU, EPT>(h1, l1, M1h, M1l, S1h);
            acc_dfh<D, MU, EPT>(h2, l2, M2h, M2l, S1h);
        }
    } else {
        const float* S1h = reinterpret_cast<const float*>(stg);
        const float* S1l = S1h + TD;
        const float* S2h = S1l + TD;
        const float* S2l = S2h + TD;
        const float* M1h = S2l + TD;
        const float* M1l = M1h + TC;
        const float* M2h = M1l + TC;
        const float* M2l = M2h + TC;
        if (kind == kApplyLaplace) {
            acc_df<D, MU, EPT>(h1, l1, M1h, M1l, S1h, S1l);
        } else if (kind == kApplyFirst) {
            acc_df<D, MU, EPT>(h1, l1, M1h, M1l, S1h, S1l);
            acc_df<D, MU, EPT>(h2, l2, M2h, M2l, S1h, S1l);
        } else if (kind == kApplyMiddle) {
            acc_df<D, MU, EPT>(h1, l1, M1h, M1l, S1h, S1l);
            acc_df<D, MU, EPT>(h2, l2, M1h, M1l, S2h, S2l);
            acc_df<D, MU, EPT>(h2, l2, M2h, M2l, S1h, S1l);
        } else {
            acc_df<D, MU, EPT>(h1, l1, M1h, M1l, S2h, S2l);
            acc_df<D, MU, EPT>(h1, l1, M2h, M2l, S1h, S1l);
        }
    }
}

template <int D, int MD, int MU = 0>
__device__ __forceinline__ void dispatch(int mu, int kind, const unsigned char* stg, double (&y1)[ApplyCfg<D, MD>::EPT],
                                         double (&y2)[ApplyCfg<D, MD>::EPT], float (&h1)[ApplyCfg<D, MD>::EPT],
                                         float (&l1)[ApplyCfg<D, MD>::EPT], float (&h2)[ApplyCfg<D, MD>::EPT],
                                         float (&l2)[ApplyCfg<D, MD>::EPT]) {
    if constexpr (MU < D) {
        if (mu == MU)
            do_job<D, MD, MU>(kind, stg, y1, y2, h1, l1, h2, l2);
        else
            dispatch<D, MD, MU + 1>(mu, kind, stg, y1, y2, h1, l1, h2, l2);
    }
}

// Block t of one apply.  The caller owns the NST staging barriers `bar`;
// uses[s] counts the phases barrier s completed before (nullptr: freshly
// initialised barriers, as for one block per CTA).
template <int D, int MD>
__device__ __forceinline__ void apply_tile(const ApplyArgs& a, const long long t, unsigned char* smem, uint64_t* bar,
                                           uint32_t* uses) {
    using C = ApplyCfg<D, MD>;
    constexpr bool DF = MD == kModeDF;
    constexpr int TE = C::TE, TD = C::TD, TC = C::TC, EPT = C::EPT;
    double* red = reinterpret_cast<double*>(smem + C::oRed);
    const int tid = threadIdx.x;
    int I[D];
#pragma unroll
    for (int mu = 0; mu < D; mu++) I[mu] = static_cast<int>((t / a.tstride[mu]) % a.nb[mu]);
    // jobs: (mode, source block J >= I_mu)
    const bool lap = a.kind == kApplyLaplace;
    int njob = 0;
    if (lap) {
#pragma unroll
        for (int mu = 0; mu < D; mu++) njob += a.nb[mu] - I[mu];
    } else {
        njob = a.nb[a.mode] - I[a.mode];
    }
    auto decode = [&](int j, int& mu, int& J) {
        if (lap) {
            mu = 0;
            while (mu < D - 1 && j >= a.nb[mu] - I[mu]) { j -= a.nb[mu] - I[mu]; mu++; }
        } else {
            mu = a.mode;
        }
        J = I[mu] + j;
    };
    const bool two_src = a.kind == kApplyMiddle || a.kind == kApplyFinal;
    const bool two_coef = !lap;
    auto issue = [&](int j, int stg) {
        int mu, J;
        decode(j, mu, J);
        const long long ts = t + static_cast<long long>(J - I[mu]) * a.tstride[mu];
        const long long tri = static_cast<long long>(J) * (J + 1) / 2 + I[mu];
        unsigned char* sb = smem + stg * C::STAGE_BYTES;
        uint32_t bytes = 0;
        if constexpr (MD == kModeF32) {
            float* S1 = reinterpret_cast<float*>(sb);
            float* S2 = S1 + 2 * TD;
            float* M1 = S1 + 4 * TD;
            float* M2 = M1 + 2 * TC;
            bytes = (two_src ? 2 : 1) * TD * 4 + (two_coef ? 2 : 1) * TC * 4;
            dev::mbar_expect_tx(&bar[stg], bytes);
            dev::bulk_g2s(S1, static_cast<const float*>(a.s1) + ts * TD, TD * 4, &bar[stg]);
            if (two_src) dev::bulk_g2s(S2, static_cast<const float*>(a.s2) + ts * TD, TD * 4, &bar[stg]);
            const float* m1 = static_cast<const float*>(lap ? a.A[mu] : a.C[mu]) + tri * TC;
            dev::bulk_g2s(M1, m1, TC * 4, &bar[stg]);
            if (two_coef) dev::bulk_g2s(M2, static_cast<const float*>(a.A[mu]) + tri * TC, TC * 4, &bar[stg]);
        } else if constexpr (MD == kModeF64) {
            double* S1 = reinterpret_cast<double*>(sb);
            double* S2 = S1 + TD;
            double* M1 = S2 + TD;
            double* M2 = M1 + TC;
            bytes = (two_src ? 2 : 1) * TD * 8 + (two_coef ? 2 : 1) * TC * 8;
            dev::mbar_expect_tx(&bar[stg], bytes);
            dev::bulk_g2s(S1, static_cast<const double*>(a.s1) + ts * TD, TD * 8, &bar[stg]);
            if (two_src) dev::bulk_g2s(S2, static_cast<const double*>(a.s2) + ts * TD, TD * 8, &bar[stg]);
            const double* m1 = static_cast<const double*>(lap ? a.A[mu] : a.C[mu]) + tri * TC;
            dev::bulk_g2s(M1, m1, TC * 8, &bar[stg]);
            if (two_coef) dev::bulk_g2s(M2, static_cast<const double*>(a.A[mu]) + tri * TC, TC * 8, &bar[stg]);
        } else if constexpr (MD == kModeDFh) {
            float* S1h = reinterpret_cast<float*>(sb);
            float* M1h = S1h + 4 * TD;
            float* M1l = M1h + TC;
            float* M2h = M1l + TC;
            float* M2l = M2h + TC;
            bytes = TD * 4 + (two_coef ? 2 : 1) * TC * 8;
            dev::mbar_expect_tx(&bar[stg], bytes);
            dev::bulk_g2s(S1h, static_cast<const float*>(a.s1) + ts * TD, TD * 4, &bar[stg]);
            const float* m1h = static_cast<const float*>(lap ? a.A[mu] : a.C[mu]) + tri * TC;
            const float* m1l = static_cast<const float*>(lap ? a.Al[mu] : a.Cl[mu]) + tri * TC;
            dev::bulk_g2s(M1h, m1h, TC * 4, &bar[stg]);
            dev::bulk_g2s(M1l, m1l, TC * 4, &bar[stg]);
            if (two_coef) {
                dev::bulk_g2s(M2h, static_cast<const float*>(a.A[mu]) + tri * TC, TC * 4, &bar[stg]);
                dev::bulk_g2s(M2l, static_cast<const float*>(a.Al[mu]) + tri * TC, TC * 4, &bar[stg]);
            }
        } else {
            float* S1h = reinterpret_cast<float*>(sb);
            float* S1l = S1h + TD;
            float* S2h = S1l + TD;
            float* S2l = S2h + TD;
            float* M1h = S2l + TD;
            float* M1l = M1h + TC;
            float* M2h = M1l + TC;
            float* M2l = M2h + TC;
            bytes = (two_src ? 2 : 1) * TD * 8 + (two_coef ? 2 : 1) * TC * 8;
            dev::mbar_expect_tx(&bar[stg], bytes);
            dev::bulk_g2s(S1h, static_cast<const float*>(a.s1) + ts * TD, TD * 4, &bar[stg]);
            dev::bulk_g2s(S1l, static_cast<const float*>(a.s1l) + ts * TD, TD * 4, &bar[stg]);
            if (two_src) {
                dev::bulk_g2s(S2h, static_cast<const float*>(a.s2) + ts * TD, TD * 4, &bar[stg]);
                dev::bulk_g2s(S2l, static_cast<const float*>(a.s2l) + ts * TD, TD * 4, &bar[stg]);
            }
            const float* m1h = static_cast<const float*>(lap ? a.A[mu] : a.C[mu]) + tri * TC;
            const float* m1l = static_cast<const float*>(lap ? a.Al[mu] : a.Cl[mu]) + tri * TC;
            dev::bulk_g2s(M1h, m1h, TC * 4, &bar[stg]);
            dev::bulk_g2s(M1l, m1l, TC * 4, &bar[stg]);
            if (two_coef) {
                dev::bulk_g2s(M2h, static_cast<const float*>(a.A[mu]) + tri * TC, TC * 4, &bar[stg]);
                dev::bulk_g2s(M2l, static_cast<const float*>(a.Al[mu]) + tri * TC, TC * 4, &bar[stg]);
            }
        }
    };
    double y1[EPT], y2[EPT];
    float h1[EPT], l1[EPT], h2[EPT], l2[EPT];
#pragma unroll
    for (int q = 0; q < EPT; q++) { y1[q] = y2[q] = 0.0; h1[q] = l1[q] = h2[q] = l2[q] = 0.f; }
    if (tid == 0) {
        for (int q = 0; q < C::NST && q < njob; q++) issue(q, q);
    }
    for (int jj = 0; jj < njob; jj++) {
        const int stg = jj % C::NST;
        const uint32_t ph = (uses ? uses[stg] : 0u) + static_cast<uint32_t>(jj / C::NST);
        const bool ok = dev::mbar_wait(&bar[stg], ph & 1u, a.timeout_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
        int mu, J;
        decode(jj, mu, J);
        dispatch<D, MD>(mu, a.kind, smem + stg * C::STAGE_BYTES, y1, y2, h1, l1, h2, l2);
        __syncthreads();
        if (tid == 0 && jj + C::NST < njob) {
            dev::fence_proxy_async();
            issue(jj + C::NST, stg);
        }
    }
    if (uses)
        for (int q = 0; q < C::NST; q++) uses[q] += static_cast<uint32_t>((njob - q + C::NST - 1) / C::NST);
    // ---- epilogue
    if (a.kind == kApplyLaplace || a.kind == kApplyFinal) {
        double ss = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int e = tid + q * kThreads;
            if ((TD % kThreads) != 0 && e >= TD) continue;
            const double v = (MD == kModeDF || MD == kModeDFh) ? df_to_double(h1[q], l1[q])
                             : MD == kModeF32 ? static_cast<double>(h1[q]) : y1[q];
            // scale given: R = B - scale * A(S) (B may be R itself: update in place)
            const double r = a.scale ? a.B[t * TD + e] - dev::step_scale(a.scale[1]) * v : a.B[t * TD + e] - v;
            a.R[t * TD + e] = r;
            ss += r * r;
            mx = fmax(mx, fabs(r));
        }
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, w);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, w));
        }
        if ((tid & 31) == 0) { red[2 * (tid >> 5)] = ss; red[2 * (tid >> 5) + 1] = mx; }
        __syncthreads();
        if (tid == 0) {
            double s2 = 0, m2 = 0;
            for (int w = 0; w < kThreads / 32; w++) { s2 += red[2 * w]; m2 = fmax(m2, red[2 * w + 1]); }
            a.part[2 * t] = s2;
            a.part[2 * t + 1] = m2;
        }
    } else {
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int e = tid + q * kThreads;
            if ((TD % kThreads) != 0 && e >= TD) continue;
            if constexpr (MD == kModeF32) {
                static_cast<float*>(a.o1)[t * TD + e] = h1[q];
                static_cast<float*>(a.o2)[t * TD + e] = h2[q];
            } else if constexpr (MD == kModeF64) {
                static_cast<double*>(a.o1)[t * TD + e] = y1[q];
                static_cast<double*>(a.o2)[t * TD + e] = y2[q];
            } else {
                float oh, ol;
                df_norm(h1[q], l1[q], oh, ol);
                static_cast<float*>(a.o1)[t * TD + e] = oh;
                static_cast<float*>(a.o1l)[t * TD + e] = ol;
                df_norm(h2[q], l2[q], oh, ol);
                static_cast<float*>(a.o2)[t * TD + e] = oh;
                static_cast<float*>(a.o2l)[t * TD + e] = ol;
            }
        }
    }
}

}  // namespace apply_detail
}  // namespace tsylv
