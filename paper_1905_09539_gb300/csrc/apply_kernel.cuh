// Operator application on the block tensor, for the residual B - A(X) of the
// refinement (and of tsylv_residual).  One CTA per output block; the block
// products along one mode (or, for the Laplace form, along every mode) are
// staged through shared memory by bulk copies exactly as in the wavefront
// kernel, but every source block J >= I_mu contributes (diagonal included)
// and nothing depends on anything else of the same launch.
//
// Two arithmetics:
//   FP64 : native double multiply-adds (FP64 pipes)
//   DF64 : every double is carried as an unevaluated float pair (hi, lo),
//          |x - hi - lo| <= 2^-48 |x|; products are formed exactly with
//          an FMA (Dekker/Veltkamp product, Ogita-Rump-Oishi "Accurate sum
//          and dot product", 2005) and accumulated with the two-sum of Knuth,
//          so the whole contraction runs on the FP32 pipes.
//
// Generalized d-term form, Horner order over the modes (one launch per mode):
//   level d-1:  P = X x C,  G = X x A
//   level l  :  P = P' x C, G = G' x C + P' x A
//   level 0  :  R = B - (G' x C + P' x A)
// Laplace form: R = B - sum_mu X x_mu A_mu in one launch.
#pragma once

#include "tsylv_internal.h"

namespace tsylv {

enum ApplyKind : int { kApplyLaplace = 0, kApplyFirst = 1, kApplyMiddle = 2, kApplyFinal = 3 };
// arithmetic of an apply: 0 FP64, 1 DF64, 2 FP32
// 3: DF64 arithmetic on FP32 sources (the source's low word is zero: the
// first refinement step's iterate s D with s a power of two)
enum ApplyMode : int { kModeF64 = 0, kModeDF = 1, kModeF32 = 2, kModeDFh = 3 };

struct ApplyArgs {
    int nb[kMaxD];
    long long tstride[kMaxD];
    long long ntiles;
    int kind;          // ApplyKind
    int mode;          // mode of the generalized level
    // sources (block tensors).  FP64: s1, s2 are double tiles.  DF64: s1h/s1l,
    // s2h/s2l are float tiles.
    const void* s1;
    const void* s1l;
    const void* s2;
    const void* s2l;
    // outputs of a generalized level (FP64: o1, o2 double; DF64: o1/o1l, o2/o2l float)
    void* o1;
    void* o1l;
    void* o2;
    void* o2l;
    const double* B;   // right-hand side (double tiles) for kApplyLaplace / kApplyFinal
    const double* scale;  // nullptr: R = B - A(X); else R = B - s A(S) with s the power of two at or
                          // above scale[1] (B may alias R)
    double* R;         // residual (double tiles)
    double* part;      // [ntiles][2]: sum of R^2, max |R| of every block
    // coefficient tiles (upper block triangle), per mode: FP64 A/C (double),
    // DF64 Ah/Al, Ch/Cl (float)
    const void* A[kMaxD];
    const void* Al[kMaxD];
    const void* C[kMaxD];
    const void* Cl[kMaxD];
    int* err;
    long long timeout_ns;
};

template <bool DF>
cudaError_t launch_apply(int d, const ApplyArgs& a, cudaStream_t s);
template <bool DF>
cudaError_t prepare_apply();
// FP32 sources and coefficient tiles, FP32 accumulation (the refinement's
// residual update from its FP32 correction).
cudaError_t launch_apply_f32(int d, const ApplyArgs& a, cudaStream_t s);
cudaError_t prepare_apply_f32();
// DF64 arithmetic on an FP32 source s1 (s1l unused), the coefficients as
// float pairs; kinds Laplace and First only (one source)
cudaError_t launch_apply_dfh(int d, const ApplyArgs& a, cudaStream_t s);
cudaError_t prepare_apply_dfh();
// One launch of many applies of order d: CTA b computes block jobs[b].y of
// the apply eqs[jobs[b].x] (device arrays).  mode: 0 FP64, 1 DF64, 2 FP32.
cudaError_t launch_apply_batched(int d, int mode, const ApplyArgs* eqs, const int2* jobs, int njobs, cudaStream_t s);
cudaError_t prepare_apply_batched();


}  // namespace tsylv
