// Dense FP64 mode products on the tensor cores: the change-of-basis
// transforms of Alg. 1 (the right-hand side into the Schur bases, the
// solution back) and of its generalized counterpart.
//
// One mode product Y = X x_mu op(M) of a column-major tensor (extents
// L x m x R around mode mu) is a batched matrix product
//     C_b (P x Q) = A_b (P x K) * B_b (K x Q),   K = m,
// either one product with A = op(M), B = X (L = 1: P = m, Q = R), or R
// products with A = X_r (L x m), B = op(M)^T (P = L, Q = m).  Every operand is
// addressed by (row stride, column stride, batch stride), so transposes cost
// nothing.  A CTA computes a 64 x 64 tile of C: the K range is staged through
// shared memory in chunks of 16 (zero-filled beyond the edges), and each of
// the four warps accumulates a 32 x 32 sub-tile as 4 x 4 tiles of the FP64
// tensor-core product mma.sync.m8n8k4 (DMMA) in registers.
#include <cstdint>

#include "tsylv_internal.h"

namespace tsylv {

namespace {

constexpr int kTP = 64;       // tile rows (P)
constexpr int kTQ = 64;       // tile columns (Q)
constexpr int kTK = 16;       // K chunk
constexpr int kPad = 68;      // shared row length: fragment loads of a half-warp hit 16 distinct banks
constexpr int kDThreads = 128;

struct GemmArgs {
    const double* A;
    const double* B;
    double* C;
    long long P, Q, K, batch;
    long long sAp, sAk, sAb;
    long long sBk, sBq, sBb;
    long long sCp, sCq, sCb;
};

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(c[0]), "+d"(c[1])
        : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kDThreads, 4) k_dmma_gemm(const GemmArgs g) {
    __shared__ double As[kTK][kPad];  // As[k][p]
    __shared__ double Bs[kTK][kPad];  // Bs[k][q]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane >> 2, ti = lane & 3;
    const int wp = (warp & 1) * 32, wq = (warp >> 1) * 32;  // the warp's 32 x 32 sub-tile
    const long long tp = (g.P + kTP - 1) / kTP, tq = (g.Q + kTQ - 1) / kTQ;
    const long long ntile = tp * tq * g.batch;
    const bool a_pfast = g.sAp == 1, b_kfast = g.sBk == 1;
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long long b = tile / (tp * tq);
        const long long rem = tile - b * tp * tq;
        const long long p0 = (rem % tp) * kTP, q0 = (rem / tp) * kTQ;
        const double* A = g.A + b * g.sAb;
        const double* B = g.B + b * g.sBb;
        double acc[4][4][2];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j][0] = acc[i][j][1] = 0.0;
        for (long long k0 = 0; k0 < g.K; k0 += kTK) {
            // stage A (64 x 16) and B (16 x 64); the index order follows the
            // unit stride so that the global loads coalesce
#pragma unroll
            for (int j = 0; j < kTP * kTK / kDThreads; j++) {
                const int idx = tid + j * kDThreads;
                const int p = a_pfast ? idx % kTP : idx / kTK;
                const int k = a_pfast ? idx / kTP : idx % kTK;
                const long long gp = p0 + p, gk = k0 + k;
                As[k][p] = (gp < g.P && gk < g.K) ? A[gp * g.sAp + gk * g.sAk] : 0.0;
                const int q = b_kfast ? idx / kTK : idx % kTQ;
                const int kb = b_kfast ? idx % kTK : idx / kTQ;
                const long long gq = q0 + q, gkb = k0 + kb;
                Bs[kb][q] = (gq < g.Q && gkb < g.K) ? B[gkb * g.sBk + gq * g.sBq] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kTK; kk += 4) {
                double af[4], bf[4];
#pragma unroll
                for (int i = 0; i < 4; i++) af[i] = As[kk + ti][wp + i * 8 + gi];  // A(row g, col t)
#pragma unroll
                for (int j = 0; j < 4; j++) bf[j] = Bs[kk + ti][wq + j * 8 + gi];  // B(row t, col g)
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) dmma(acc[i][j], af[i], bf[j]);
            }
            __syncthreads();
        }
        double* C = g.C + b * g.sCb;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const long long p = p0 + wp + i * 8 + gi, q = q0 + wq + j * 8 + 2 * ti + h;  // C(row g, col 2t+h)
                    if (p < g.P && q < g.Q) C[p * g.sCp + q * g.sCq] = acc[i][j][h];
                }
    }
}

int g_dmma_grid[64] = {};

int dmma_grid() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * 4;
    if (!g_dmma_grid[dev]) {
        int sms = 0, occ = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dmma_gemm, kDThreads, 0) != cudaSuccess || occ < 1)
            occ = 4;
        (void)cudaGetLastError();
        g_dmma_grid[dev] = sms * occ;
    }
    return g_dmma_grid[dev];
}

}  // namespace

// Y = X x_mu op(M) for a column-major tensor of extents (L, m, R) around mode
// mu; op(M) = M^T when trans.  X and Y must not alias.
cudaError_t launch_dmma_modeprod(const double* X, const double* M, bool trans, double* Y, long long L, long long m,
                                 long long R, cudaStream_t s) {
    GemmArgs g{};
    g.K = m;
    const long long sMi = trans ? m : 1, sMk = trans ? 1 : m;  // op(M)(i, k) = M[i * sMi + k * sMk]
    if (L == 1) {
        g.A = M; g.sAp = sMi; g.sAk = sMk; g.sAb = 0;
        g.B = X; g.sBk = 1; g.sBq = m; g.sBb = 0;
        g.C = Y; g.sCp = 1; g.sCq = m; g.sCb = 0;
        g.P = m; g.Q = R; g.batch = 1;
    } else {
        g.A = X; g.sAp = 1; g.sAk = L; g.sAb = L * m;
        g.B = M; g.sBk = sMk; g.sBq = sMi; g.sBb = 0;   // B(k, i) = op(M)(i, k)
        g.C = Y; g.sCp = 1; g.sCq = L; g.sCb = L * m;
        g.P = L; g.Q = m; g.batch = R;
    }
    const long long ntile = ((g.P + kTP - 1) / kTP) * ((g.Q + kTQ - 1) / kTQ) * g.batch;
    const long long cap = dmma_grid();
    const int grid = static_cast<int>(ntile < cap ? ntile : cap);
    k_dmma_gemm<<<grid, kDThreads, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace tsylv
