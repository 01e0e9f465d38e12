// Adjoint kernels (tsylv_backward).
#pragma once

#include "tsylv_internal.h"

namespace tsylv {

// Y = X x_mu M (M n x n upper quasi-triangular if quasi, else upper
// triangular); X, Y column-major with the mode-mu matricization of L x n x R.
cudaError_t launch_modeprod(const double* X, const double* M, double* Y, long long L, int n, long long R, bool quasi,
                            cudaStream_t s);
// G += Lm_(mu) W_(mu)^T on the quasi-upper part (G must be zeroed first).
cudaError_t launch_gram(const double* Lm, const double* W, double* G, long long L, int n, long long R, cudaStream_t s);
// out = -mask(G) (mask of A: quasi-upper pattern of A; of C: upper triangle).
cudaError_t launch_finalize_grad(const double* G, const double* A, double* out, int n, bool is_c, cudaStream_t s);

}  // namespace tsylv
