// Mixed-precision refinement: declarations shared by the host driver and
// its kernels.
#pragma once

#include "apply_kernel.cuh"
#include "tsylv_internal.h"

namespace tsylv {

struct NormArgs {
    const double* M[2 * kMaxD];
    int n[2 * kMaxD];
    int upper[2 * kMaxD];
};

cudaError_t launch_tile_stats(const double* x, double* part, long long nt, int td, cudaStream_t s);
cudaError_t launch_split(const double* x, float* h, float* l, long long n, cudaStream_t s);
cudaError_t prepare_norm2();  // shared-memory limit of the norm estimate (before any capture)
cudaError_t launch_scale_to_f32(const double* r, float* r32, const double* nrm, long long n, cudaStream_t s);
cudaError_t launch_update_x(double* x, const float* d32, const double* nrm, float* xh, float* xl, double* xpart,
                            long long n, int td, cudaStream_t s);
cudaError_t launch_reduce(const double* part, const double* xpart, long long nt, double* nrm, cudaStream_t s);
cudaError_t launch_norm2(const NormArgs& a, int count, int nmax, double* out, cudaStream_t s);

}  // namespace tsylv
