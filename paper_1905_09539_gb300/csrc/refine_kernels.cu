// Elementwise and reduction kernels of the mixed-precision refinement:
// scaling of the residual into the FP32 solve, the FP64 correction update of
// X, double -> float-pair splitting for the DF64 residual, norm reductions and
// spectral-norm estimates of the coefficients.
#include "device_common.cuh"
#include "refine.h"

namespace tsylv {

namespace {

inline int grid_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

// x (double) -> (hi, lo) floats with hi + lo = x to 2^-48 relative
__global__ void k_split(const double* __restrict__ x, float* __restrict__ h, float* __restrict__ l, long long n) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double v = x[i];
        const float hv = static_cast<float>(v);
        h[i] = hv;
        l[i] = static_cast<float>(v - static_cast<double>(hv));
    }
}

// r32 = r64 / s, s = the power of two at or above max|r64| (read from the
// device-side norm record)
__global__ void k_scale_to_f32(const double* __restrict__ r, float* __restrict__ r32, const double* __restrict__ nrm,
                               long long n) {
    const double s = 1.0 / dev::step_scale(nrm[1]);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        r32[i] = static_cast<float>(r[i] * s);
}

// x += s * d32 (the correction of the scaled system), optional split of
// the new x, and per-block partial sums of x^2 into part[2*blk + 0] (the
// residual kernels own part[.. + 0, 1] of another array).
__global__ void k_update_x(double* __restrict__ x, const float* __restrict__ d32, const double* __restrict__ nrm,
                           float* __restrict__ xh, float* __restrict__ xl, double* __restrict__ xpart, long long n,
                           int td) {
    const double s = dev::step_scale(nrm[1]);
    for (long long blk = blockIdx.x; blk * td < n; blk += gridDim.x) {
        double ss = 0;
        for (int e = threadIdx.x; e < td; e += blockDim.x) {
            const long long i = blk * td + e;
            const double v = x[i] + s * static_cast<double>(d32[i]);
            x[i] = v;
            if (xh) {
                const float hv = static_cast<float>(v);
                xh[i] = hv;
                xl[i] = static_cast<float>(v - static_cast<double>(hv));
            }
            ss += v * v;
        }
        for (int w = 16; w >= 1; w >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, w);
        __shared__ double red[32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); w++) t += red[w];
            xpart[blk] = t;
        }
        __syncthreads();
    }
}

// nrm[0] = sum part[2i], nrm[1] = max part[2i+1], nrm[2] = sum xpart[i]
__global__ void k_reduce(const double* __restrict__ part, const double* __restrict__ xpart, long long nt,
                         double* __restrict__ nrm) {
    double s = 0, m = 0, x = 0;
    for (long long i = threadIdx.x; i < nt; i += blockDim.x) {
        s += part[2 * i];
        m = fmax(m, part[2 * i + 1]);
        if (xpart) x += xpart[i];
    }
    for (int w = 16; w >= 1; w >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, w);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, w));
        x += __shfl_xor_sync(0xffffffffu, x, w);
    }
    __shared__ double red[3][32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s;
        red[1][threadIdx.x >> 5] = m;
        red[2][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); w++) {
            a += red[0][w];
            b = fmax(b, red[1][w]);
            c += red[2][w];
        }
        nrm[0] = a;
        nrm[1] = b;
        nrm[2] = c;
    }
}

// ||M||_2 estimate of an n x n column-major matrix (structural zeros below
// the first subdiagonal ignored): 30 steps of power iteration on M^T M in
// FP32, one CTA per matrix.  The estimate only scales the stopping test.
// When it fits (n <= kNormSmemN) the matrix is first staged in shared memory
// as floats, packed by columns (upper triangle, entry (i, j), i <= j, at
// j (j + 1) / 2 + i) plus the first subdiagonal, so that the iterations read
// no global memory; larger matrices are read from global memory.
constexpr int kNormSmemN = 320;
constexpr size_t norm_smem_bytes(int n) {
    return (static_cast<size_t>(n) * (n + 1) / 2 + 3 * static_cast<size_t>(n)) * sizeof(float);
}

__global__ void k_norm2(NormArgs a, double* __restrict__ out) {
    const int mat = blockIdx.x;
    const double* M = a.M[mat];
    const int n = a.n[mat];
    const int upper = a.upper[mat];
    extern __shared__ float shf[];
    float* v = shf;          // n
    float* w = shf + n;      // n
    const bool staged = n <= kNormSmemN;
    float* sub = shf + 2 * n;  // n: M(j + 1, j)
    float* P = shf + 3 * n;    // packed upper triangle
    __shared__ float red[32];
    if (staged) {
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {  // coalesced, independent loads
            const int i = idx % n, j = idx / n;
            if (i <= j) P[static_cast<size_t>(j) * (j + 1) / 2 + i] = static_cast<float>(M[idx]);
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            sub[j] = (!upper && j + 1 < n) ? static_cast<float>(M[j + 1 + static_cast<long long>(n) * j]) : 0.f;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.0f + 0.01f * (i % 7);
    __syncthreads();
    float lam = 0.f;
    for (int it = 0; it < 30; it++) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {  // w = M v
            float s = 0.f;
            if (staged) {
                if (i > 0) s = sub[i - 1] * v[i - 1];
                for (int j = i; j < n; j++) s = fmaf(P[static_cast<size_t>(j) * (j + 1) / 2 + i], v[j], s);
            } else {
                const int j0 = upper ? i : (i > 0 ? i - 1 : 0);
                for (int j = j0; j < n; j++) s = fmaf(static_cast<float>(M[i + static_cast<long long>(n) * j]), v[j], s);
            }
            w[i] = s;
        }
        __syncthreads();
        float part = 0.f;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {  // v = M^T w
            float s = 0.f;
            if (staged) {
                const float* col = P + static_cast<size_t>(j) * (j + 1) / 2;
                for (int i = 0; i <= j; i++) s = fmaf(col[i], w[i], s);
                if (j + 1 < n) s = fmaf(sub[j], w[j + 1], s);
            } else {
                const int iend = upper ? j : (j + 1 < n ? j + 1 : n - 1);
                for (int i = 0; i <= iend; i++) s = fmaf(static_cast<float>(M[i + static_cast<long long>(n) * j]), w[i], s);
            }
            v[j] = s;
            part += s * s;
        }
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int q = 0; q < static_cast<int>(blockDim.x >> 5); q++) t += red[q];
            red[31] = sqrtf(t);
        }
        __syncthreads();
        const float nv = red[31];
        lam = nv;
        const float inv = nv > 0.f ? 1.0f / nv : 0.f;
        for (int j = threadIdx.x; j < n; j += blockDim.x) v[j] *= inv;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[mat] = sqrt(static_cast<double>(lam));
}

// part[2 t] = sum x^2, part[2 t + 1] = max |x| over block t
__global__ void k_tile_stats(const double* __restrict__ x, double* __restrict__ part, long long nt, int td) {
    for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
        double ss = 0, mx = 0;
        for (int e = threadIdx.x; e < td; e += blockDim.x) {
            const double v = x[t * td + e];
            ss += v * v;
            mx = fmax(mx, fabs(v));
        }
        for (int w = 16; w >= 1; w >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, w);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, w));
        }
        __shared__ double red[2][32];
        if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ss; red[1][threadIdx.x >> 5] = mx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); w++) { a += red[0][w]; b = fmax(b, red[1][w]); }
            part[2 * t] = a;
            part[2 * t + 1] = b;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_tile_stats(const double* x, double* part, long long nt, int td, cudaStream_t s) {
    int g = static_cast<int>(nt < 152LL * 16 ? nt : 152LL * 16);
    if (g < 1) g = 1;
    k_tile_stats<<<g, 128, 0, s>>>(x, part, nt, td);
    return cudaGetLastError();
}

cudaError_t launch_split(const double* x, float* h, float* l, long long n, cudaStream_t s) {
    k_split<<<grid_for(n), 256, 0, s>>>(x, h, l, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_to_f32(const double* r, float* r32, const double* nrm, long long n, cudaStream_t s) {
    k_scale_to_f32<<<grid_for(n), 256, 0, s>>>(r, r32, nrm, n);
    return cudaGetLastError();
}

cudaError_t launch_update_x(double* x, const float* d32, const double* nrm, float* xh, float* xl, double* xpart,
                            long long n, int td, cudaStream_t s) {
    long long nb = n / td;
    int g = static_cast<int>(nb < 152LL * 16 ? nb : 152LL * 16);
    if (g < 1) g = 1;
    k_update_x<<<g, 128, 0, s>>>(x, d32, nrm, xh, xl, xpart, n, td);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* part, const double* xpart, long long nt, double* nrm, cudaStream_t s) {
    k_reduce<<<1, 1024, 0, s>>>(part, xpart, nt, nrm);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const NormArgs& a, int count, int nmax, double* out, cudaStream_t s) {
    const size_t sm = nmax <= kNormSmemN ? norm_smem_bytes(nmax) : 2 * static_cast<size_t>(nmax) * sizeof(float);
    k_norm2<<<count, 256, sm, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t prepare_norm2() {
    return cudaFuncSetAttribute(k_norm2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(norm_smem_bytes(kNormSmemN)));
}

}  // namespace tsylv
