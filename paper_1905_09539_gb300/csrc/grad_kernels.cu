// Kernels of the adjoint (tsylv_backward): mode products of column-major
// tensors with (quasi-)triangular coefficients, the masked gradient
// contraction G = L_(mu) W_(mu)^T, and the final masking/negation.
#include "grad.h"

namespace tsylv {

namespace {

// Y = X x_mu M with M upper quasi-triangular (quasi = 1) or upper triangular:
// Y(.., i, ..) = sum_{k >= i - quasi} M(i, k) X(.., k, ..).  FP64.
__global__ void k_modeprod(const double* __restrict__ X, const double* __restrict__ M, double* __restrict__ Y,
                           long long L, int n, long long R, int quasi) {
    const long long total = L * n * R;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long l = idx % L;
        const long long rest = idx / L;
        const int i = static_cast<int>(rest % n);
        const long long r = rest / n;
        const double* xs = X + l + L * n * r;
        int k0 = i - quasi;
        if (k0 < 0) k0 = 0;
        if (quasi && k0 < i && M[i + static_cast<long long>(n) * k0] == 0.0) k0 = i;
        double s0 = 0, s1 = 0;
        int k = k0;
        for (; k + 1 < n; k += 2) {
            s0 = fma(M[i + static_cast<long long>(n) * k], xs[L * k], s0);
            s1 = fma(M[i + static_cast<long long>(n) * (k + 1)], xs[L * (k + 1)], s1);
        }
        if (k < n) s0 = fma(M[i + static_cast<long long>(n) * k], xs[L * k], s0);
        Y[idx] = s0 + s1;
    }
}

// G(i, j) += sum_p Lm(i, p) W(j, p) over the mode-mu matricizations, for the
// 32 x 32 output tile (bi, bj) and the contraction chunk kz of K = L * R.
// Tiles entirely below the first subdiagonal are skipped (masked anyway).
constexpr int GT = 32;   // output tile
constexpr int GK = 32;   // contraction chunk staged per step
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ Lm, const double* __restrict__ W,
                                              double* __restrict__ G, long long L, int n, long long R,
                                              long long kchunk) {
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bi * GT > bj * GT + GT) return;  // below the subdiagonal: masked
    const long long K = L * R;
    const long long kb = blockIdx.z * kchunk;
    const long long ke = kb + kchunk < K ? kb + kchunk : K;
    __shared__ double sa[GK][GT + 1];
    __shared__ double sb[GK][GT + 1];
    const int tid = threadIdx.x;
    const int ti = tid % 16, tj = tid / 16;  // each thread: 2 x 2 outputs
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (long long p0 = kb; p0 < ke; p0 += GK) {
        for (int q = tid; q < GK * GT; q += 256) {
            const int pp = q / GT, ii = q % GT;
            const long long p = p0 + pp;
            const int gi = bi * GT + ii, gj = bj * GT + ii;
            double va = 0, vb = 0;
            if (p < ke) {
                const long long l = p % L, r = p / L;
                const long long base = l + L * static_cast<long long>(n) * r;
                if (gi < n) va = Lm[base + L * gi];
                if (gj < n) vb = W[base + L * gj];
            }
            sa[pp][ii] = va;
            sb[pp][ii] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int pp = 0; pp < GK; pp++) {
            const double a0 = sa[pp][ti], a1 = sa[pp][ti + 16];
            const double b0 = sb[pp][tj], b1 = sb[pp][tj + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
        for (int y = 0; y < 2; y++) {
            const int gi = bi * GT + ti + 16 * x, gj = bj * GT + tj + 16 * y;
            if (gi < n && gj < n && gi <= gj + 1) atomicAdd(&G[gi + static_cast<long long>(n) * gj], acc[x][y]);
        }
}

// out = -mask(G): mask_A keeps i <= j and the subdiagonal entries of the
// 2x2 blocks of A (A(i, i-1) != 0); mask_C keeps i <= j.
__global__ void k_finalize(const double* __restrict__ G, const double* __restrict__ A, double* __restrict__ out, int n,
                           int is_c) {
    const long long total = static_cast<long long>(n) * n;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(idx % n), j = static_cast<int>(idx / n);
        bool keep = i <= j;
        if (!is_c && i == j + 1) keep = A[idx] != 0.0;
        out[idx] = keep ? -G[idx] : 0.0;
    }
}

inline int grid_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

}  // namespace

cudaError_t launch_modeprod(const double* X, const double* M, double* Y, long long L, int n, long long R, bool quasi,
                            cudaStream_t s) {
    k_modeprod<<<grid_for(L * n * R), 256, 0, s>>>(X, M, Y, L, n, R, quasi ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_gram(const double* Lm, const double* W, double* G, long long L, int n, long long R, cudaStream_t s) {
    const int nt = (n + GT - 1) / GT;
    const long long K = L * R;
    // enough contraction chunks to give every SM a few CTAs
    long long chunks = (152LL * 8 + nt * nt - 1) / (nt * nt);
    if (chunks < 1) chunks = 1;
    long long kchunk = (K + chunks - 1) / chunks;
    kchunk = (kchunk + GK - 1) / GK * GK;
    chunks = (K + kchunk - 1) / kchunk;
    if (chunks > 65535) {
        chunks = 65535;
        kchunk = ((K + chunks - 1) / chunks + GK - 1) / GK * GK;
        chunks = (K + kchunk - 1) / kchunk;
    }
    dim3 grid(nt, nt, static_cast<unsigned>(chunks));
    k_gram<<<grid, 256, 0, s>>>(Lm, W, G, L, n, R, kchunk);
    return cudaGetLastError();
}

cudaError_t launch_finalize_grad(const double* G, const double* A, double* out, int n, bool is_c, cudaStream_t s) {
    k_finalize<<<grid_for(static_cast<long long>(n) * n), 256, 0, s>>>(G, A, out, n, is_c ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace tsylv
