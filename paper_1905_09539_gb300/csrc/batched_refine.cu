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

// r32 = r / s_e, s_e the power of two at or above max|r_e| (nrm[4 e + 1])
__global__ void k_bscale(const double* __restrict__ r, float* __restrict__ r32, const int* __restrict__ tile_eq,
                         const double* __restrict__ nrm, long long n, int td) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        r32[i] = static_cast<float>(r[i] * (1.0 / dev::step_scale(nrm[4 * tile_eq[i / td] + 1])));
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

// ||M||_2 estimates of many n x n column-major matrices (one CTA each): 30
// steps of power iteration on M^T M in FP32 over the structurally nonzero
// part (upper triangle, plus the first subdiagonal when upper == 0).  The
// estimates only scale the stopping test.
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
                const int j0 = up ? i : (i > 0 ? i - 1 : 0);
                for (int j = j0; j < n; j++) s = fmaf(static_cast<float>(M[i + static_cast<long long>(n) * j]), v[j], s);
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
    k_bscale<<<grid_for(n), 256, 0, s>>>(r, r32, tile_eq, nrm, n, td);
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
    const int g = count < 152 * 8 ? count : 152 * 8;
    k_bnorm2<<<g > 0 ? g : 1, 256, 2 * nmax * sizeof(float), s>>>(pool, off, nmat, upper, count, out);
    return cudaGetLastError();
}

}  // namespace tsylv
