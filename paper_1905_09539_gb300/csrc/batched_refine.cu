// Elementwise and reduction kernels of the batched mixed-precision
// refinement.  Every pool holds the block tensors of all equations back to
// back (equation e owns the blocks [tile_off[e], tile_off[e+1]) of td entries
// each); per-equation scalars are indexed through the block -> equation map.
#include "batched.h"
#include "device_common.cuh"

namespace tsylv {

namespace {

inline int grid_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

// r32 = r / s_e, s_e the power of two at or above max|r_e| (nrm[4 e + 1]):
// one CTA per block at a time, the exact reciprocal of s_e taken once per block
__global__ void k_bscale(const double* __restrict__ r, float* __restrict__ r32, const int* __restrict__ tile_eq,
                         const double* __restrict__ nrm, long long ntiles, int td) {
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const double inv = 1.0 / dev::step_scale(nrm[4 * tile_eq[t] + 1]);  // a power of two: exact
        const double* rt = r + t * td;
        float* ot = r32 + t * td;
        for (int e = threadIdx.x; e < td; e += blockDim.x) ot[e] = static_cast<float>(rt[e] * inv);
    }
}

// x += s_e d32 per block, and the block's sum of x^2
__global__ void k_bupdate(double* __restrict__ x, const float* __restrict__ d32, const int* __restrict__ tile_eq,
                          const double* __restrict__ nrm, double* __restrict__ xpart, long long ntiles, int td) {
    __shared__ double red[32];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const double sc = dev::step_scale(nrm[4 * tile_eq[t] + 1]);
        double ss = 0;
        for (int e = threadIdx.x; e < td; e += blockDim.x) {
            const long long i = t * td + e;
            const double v = x[i] + sc * static_cast<double>(d32[i]);
            x[i] = v;
            ss += v * v;
        }
        for (int w = 16; w >= 1; w >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, w);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); w++) s += red[w];
            xpart[t] = s;
        }
        __syncthreads();
    }
}

// per equation e (one CTA): nrm[4e] = sum part[2t], nrm[4e+1] = max part[2t+1],
// nrm[4e+2] = sum xpart[t] over its blocks (xpart may be nullptr)
__global__ void k_breduce(const double* __restrict__ part, const double* __restrict__ xpart,
                          const long long* __restrict__ tile_off, int count, double* __restrict__ nrm) {
    __shared__ double red[3][32];
    for (int e = blockIdx.x; e < count; e += gridDim.x) {
        double s = 0, m = 0, x = 0;
        for (long long t = tile_off[e] + threadIdx.x; t < tile_off[e + 1]; t += blockDim.x) {
            s += part[2 * t];
            m = fmax(m, part[2 * t + 1]);
            if (xpart) x += xpart[t];
        }
        for (int w = 16; w >= 1; w >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, w);
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, w));
            x += __shfl_xor_sync(0xffffffffu, x, w);
        }
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
            nrm[4 * e] = a;
            nrm[4 * e + 1] = b;
            nrm[4 * e + 2] = c;
        }
        __syncthreads();
    }
}

// ||M||_2 estimates of many n x n column-major matrices: 30 steps of power
// iteration on M^T M in FP32 over the structurally nonzero part (upper
// triangle, plus the first subdiagonal when upper == 0).  The estimates only
// scale the stopping test.
//   k_bnorm2_warp: n <= kNormWarpN, one warp per matrix, the matrix held in
//   shared memory as floats (the batch's small equations);
//   k_bnorm2: any n, one CTA per matrix, reading the matrix from memory.
constexpr int kNormWarpN = 48;  // four warps' matrices within 48 KB of shared memory
constexpr int kNormWarps = 4;

__device__ __forceinline__ int norm_j0(int i, int up) { return up ? i : (i > 0 ? i - 1 : 0); }

__global__ void __launch_bounds__(32 * kNormWarps) k_bnorm2_warp(const double* __restrict__ pool,
                                                                 const long long* __restrict__ off,
                                                                 const long long* __restrict__ nmat,
                                                                 const int* __restrict__ upper, int count,
                                                                 int nmax, double* __restrict__ out) {
    extern __shared__ float shw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* Ms = shw + static_cast<size_t>(wid) * (nmax * nmax + 2 * nmax);
    float* v = Ms + nmax * nmax;
    float* w = v + nmax;
    for (int mat = blockIdx.x * kNormWarps + wid; mat < count; mat += gridDim.x * kNormWarps) {
        const double* M = pool + off[mat];
        const int n = static_cast<int>(nmat[mat]);
        const int up = upper[mat];
        for (int k = lane; k < n * n; k += 32) Ms[k] = static_cast<float>(M[k]);
        for (int i = lane; i < n; i += 32) v[i] = 1.0f + 0.01f * (i % 7);
        __syncwarp();
        float lam = 0.f;
        for (int it = 0; it < 30; it++) {
            for (int i = lane; i < n; i += 32) {  // w = M v
                float acc = 0.f;
                for (int j = norm_j0(i, up); j < n; j++) acc = fmaf(Ms[i + n * j], v[j], acc);
                w[i] = acc;
            }
            __syncwarp();
            float part = 0.f;
            for (int j = lane; j < n; j += 32) {  // v = M^T w
                float acc = 0.f;
                const int iend = up ? j : (j + 1 < n ? j + 1 : n - 1);
                for (int i = 0; i <= iend; i++) acc = fmaf(Ms[i + n * j], w[i], acc);
                v[j] = acc;
                part += acc * acc;
            }
            for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const float nv = sqrtf(part);
            lam = nv;
            const float inv = nv > 0.f ? 1.0f / nv : 0.f;
            __syncwarp();
            for (int j = lane; j < n; j += 32) v[j] *= inv;
            __syncwarp();
        }
        if (lane == 0) out[mat] = sqrt(static_cast<double>(lam));
        __syncwarp();
    }
}

__global__ void k_bnorm2(const double* __restrict__ pool, const long long* __restrict__ off,
                         const long long* __restrict__ nmat, const int* __restrict__ upper, int count,
                         double* __restrict__ out) {
    extern __shared__ float shf[];
    __shared__ float red[32];
    for (int mat = blockIdx.x; mat < count; mat += gridDim.x) {
        const double* M = pool + off[mat];
        const int n = static_cast<int>(nmat[mat]);
        const int up = upper[mat];
        float* v = shf;
        float* w = shf + n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.0f + 0.01f * (i % 7);
        __syncthreads();
        float lam = 0.f;
        for (int it = 0; it < 30; it++) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                float s = 0.f;
                for (int j = norm_j0(i, up); j < n; j++) s = fmaf(static_cast<float>(M[i + static_cast<long long>(n) * j]), v[j], s);
                w[i] = s;
            }
            __syncthreads();
            float part = 0.f;
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                float s = 0.f;
                const int iend = up ? j : (j + 1 < n ? j + 1 : n - 1);
                for (int i = 0; i <= iend; i++) s = fmaf(static_cast<float>(M[i + static_cast<long long>(n) * j]), w[i], s);
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
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_bscale(const double* r, float* r32, const int* tile_eq, const double* nrm, long long n, int td,
                          cudaStream_t s) {
    const long long ntiles = n / td;
    const int g = static_cast<int>(ntiles < 152LL * 16 ? (ntiles > 0 ? ntiles : 1) : 152LL * 16);
    k_bscale<<<g, 128, 0, s>>>(r, r32, tile_eq, nrm, ntiles, td);
    return cudaGetLastError();
}

cudaError_t launch_bupdate(double* x, const float* d32, const int* tile_eq, const double* nrm, double* xpart,
                           long long ntiles, int td, cudaStream_t s) {
    const int g = static_cast<int>(ntiles < 152LL * 16 ? (ntiles > 0 ? ntiles : 1) : 152LL * 16);
    k_bupdate<<<g, 128, 0, s>>>(x, d32, tile_eq, nrm, xpart, ntiles, td);
    return cudaGetLastError();
}

cudaError_t launch_breduce(const double* part, const double* xpart, const long long* tile_off, int count, double* nrm,
                           cudaStream_t s) {
    const int g = count < 152 * 8 ? count : 152 * 8;
    k_breduce<<<g > 0 ? g : 1, 256, 0, s>>>(part, xpart, tile_off, count, nrm);
    return cudaGetLastError();
}

cudaError_t launch_bnorm2(const double* pool, const long long* off, const long long* nmat, const int* upper, int count,
                          long long nmax, double* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (nmax <= kNormWarpN) {
        const int nm = static_cast<int>(nmax);
        const size_t sm = static_cast<size_t>(kNormWarps) * (nm * nm + 2 * nm) * sizeof(float);
        const int g = (count + kNormWarps - 1) / kNormWarps;
        k_bnorm2_warp<<<g, 32 * kNormWarps, sm, s>>>(pool, off, nmat, upper, count, nm, out);
        return cudaGetLastError();
    }
    const int g = count < 152 * 8 ? count : 152 * 8;
    k_bnorm2<<<g, 256, 2 * nmax * sizeof(float), s>>>(pool, off, nmat, upper, count, out);
    return cudaGetLastError();
}

}  // namespace tsylv
