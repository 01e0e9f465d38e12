// Dense mode transforms Y = X x_1 op(M_1) x_2 ... x_d op(M_d) of column-major
// tensors: the orthogonal changes of basis of Alg. 1 (right-hand side in,
// solution out) and of its generalized counterpart (Sec. 3, the Q and Z factors of the
// generalized Schur forms), which take an equation with general coefficients
// to the (quasi-)triangular one the solver handles and its solution back.
// Dense FP64 mode products on the tensor cores (DMMA, dmma_modeprod.cu).
#include <cstring>

#include "solver.h"
#include "tsylv_internal.h"

namespace tsylv {

cudaError_t launch_dmma_modeprod(const double* X, const double* M, bool trans, double* Y, long long L, long long m,
                                 long long R, cudaStream_t s);

namespace {

bool dims_ok(int d, const int64_t* n, long long* N) {
    if (d < 1 || d > kMaxD || !n) return false;
    long long t = 1;
    for (int mu = 0; mu < d; mu++) {
        if (n[mu] < 1 || n[mu] > (1 << 20)) return false;
        t *= n[mu];
        if (t > (1LL << 34)) return false;
    }
    *N = t;
    return true;
}

}  // namespace

size_t transform_workspace_bytes(int d, const int64_t* n) {
    long long N = 0;
    if (!dims_ok(d, n, &N)) return 0;
    return static_cast<size_t>(N) * sizeof(double) + 256;
}

// Y(.., i_mu, ..) = sum_k op(M_mu)(i_mu, k) X(.., k, ..) applied mode after
// mode.  For mode mu the tensor is R = prod_{eta > mu} n_eta column-major
// L x n_mu matrices (L = prod_{eta < mu} n_eta) and each becomes X_r op(M)^T;
// for L = 1 the whole mode is the single product op(M) X (n_mu x R).  Every
// product runs in the project's DMMA kernel (no library GEMM).
int transform(int d, const int64_t* n, const double* const* M, const int* trans, const double* X, double* Y,
              void* work, size_t work_bytes, cudaStream_t stream) {
    long long N = 0;
    if (!dims_ok(d, n, &N)) return d < 1 || d > kMaxD ? -1 : -2;
    if (!M) return -3;
    if (!X) return -5;
    if (!Y) return -6;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -7;
    if (work_bytes < transform_workspace_bytes(d, n)) return -8;
    int active[kMaxD], na = 0;
    for (int mu = 0; mu < d; mu++)
        if (M[mu] != nullptr) active[na++] = mu;
    cudaError_t e;
    if (na == 0) {
        if (X != Y && (e = cudaMemcpyAsync(Y, X, static_cast<size_t>(N) * 8, cudaMemcpyDeviceToDevice, stream)) !=
                          cudaSuccess)
            return cuda_fail(e, "transform: copy");
        return TSYLV_OK;
    }
    double* tmp = static_cast<double*>(work);
    // products alternate between tmp and Y so that the last one writes Y;
    // the first reads X, which may alias Y: then it writes tmp and an odd
    // count ends with a copy
    const bool alias = X == Y;
    const double* src = X;
    for (int j = 0; j < na; j++) {
        const int mu = active[j];
        double* dst;
        if (alias)
            dst = (j % 2 == 0) ? tmp : Y;
        else
            dst = ((na - 1 - j) % 2 == 0) ? Y : tmp;
        long long L = 1, R = 1;
        for (int eta = 0; eta < mu; eta++) L *= n[eta];
        for (int eta = mu + 1; eta < d; eta++) R *= n[eta];
        if ((e = launch_dmma_modeprod(src, M[mu], trans && trans[mu], dst, L, n[mu], R, stream)) != cudaSuccess)
            return cuda_fail(e, "transform: mode product");
        src = dst;
    }
    if (src != Y) {
        if ((e = cudaMemcpyAsync(Y, src, static_cast<size_t>(N) * 8, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
            return cuda_fail(e, "transform: copy");
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "transform");
    return TSYLV_OK;
}

}  // namespace tsylv
