// Pipelined first two refinement steps of the Laplace form: launch
// declarations.
#pragma once

#include "apply_kernel.cuh"
#include "batched.h"

namespace tsylv {

// First two refinement steps of the Laplace form in one launch, pipelined
// over the blocks: queue jobs (kind << 26 | block), kinds
//   0  S1: FP32 solve of the block (R0 / s in w1.X, D1 out), flag s1done
//   1  R1: R1 = B - s A(D1) on the block in double-float arithmetic, then the
//          block's right-hand side R1 / s of the second solve (w2.X), flag r1done
//   2  S2: FP32 solve of the block (w2.X: R1 / s in, D2 out), flag w2.ready
//   3  R2: R2 = R1 - s A(D2) on the block in FP32 (the residual update)
// Every job waits only for jobs earlier in the queue (R1 of a block for its
// S1, S2 for its R1 and the S2 of its sources, R2 for its S2), so progress
// needs no co-residency.  s = the scale of the first step (nrm[1]) for both
// solves: both scalings are exact, so the result equals two separate steps.
struct Refine2Args {
    const WaveArgs* w1;   // device parameter blocks of the two solves (ready = s1done / s2done)
    const WaveArgs* w2;
    const int* jobs;
    int njobs;
    int* head;            // queue head
    int* abort;
    long long timeout_ns;
    int* r1done;          // per block: R1 and the second right-hand side written
    ApplyArgs r1;         // kind Laplace, DF64 on the float source D1, scale nrm
    ApplyArgs r2;         // kind Laplace, FP32 update R -= s A(D2), scale nrm
    float* X2;            // w2's block tensor (right-hand side / solution of the second solve)
    const double* nrm;
};

// prod (ProductKind): arithmetic of the FP32 solves' block updates.
cudaError_t launch_refine2(int d, int prod, const Refine2Args& f, int grid, cudaStream_t s);
int refine2_occupancy(int d, int prod);
cudaError_t prepare_refine2();

}  // namespace tsylv
