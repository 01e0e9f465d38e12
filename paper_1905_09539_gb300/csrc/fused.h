// Fused first refinement step (FP32 solve + FP64 update + DF64 residual) of
// the Laplace form: launch declarations.
#pragma once

#include "apply_kernel.cuh"
#include "batched.h"

namespace tsylv {

struct FusedArgs {
    BatchArgs b;          // one equation's blocks in wavefront order (jobs == nullptr)
    ApplyArgs ap;         // the DF64 residual (kind Laplace) of every block
    double* X;            // FP64 block tensor of the iterate
    float* Xh;            // its float-pair split
    float* Xl;
    double* xpart;        // per-block sums of X^2
    const double* nrm;    // nrm[1]: scale s of the step
    int lag;              // residual job i follows solve job i + lag in the queue
};


cudaError_t launch_fused(int d, const FusedArgs& f, int grid, cudaStream_t s);
cudaError_t prepare_fused();
int fused_occupancy(int d);

}  // namespace tsylv
