// Batched solve of many independent equations: declarations shared by the
// host driver (batched.cpp) and its kernels.
//
// Every equation keeps the block grid of a single solve (block tensor,
// coefficient tiles, partition tables).  One persistent launch works through
// a job queue holding every block of every equation; before a block reads a
// source block for its update it waits until that block's "solved" flag is
// set (optionally, a job may also wait for a count of finished blocks of its
// equation).  Jobs are queued so that every block's sources sit earlier in the
// queue; a CTA that waits therefore only waits on jobs that running CTAs
// already hold, and the launch needs no co-residency guarantee.  The single
// solve uses the same kernel with a queue of one equation's blocks.
#pragma once

#include "tsylv_internal.h"

namespace tsylv {

struct BatchJob {
    int eq;      // equation
    int tile;    // linear block index in the equation's block grid
    int need;    // blocks of equation `eq` that must be finished first
    int pad;
};

// Per-equation geometry of the layout kernels (pools are kernel arguments).
struct BatchGeom {
    int d;
    int nb[kMaxD];
    long long n[kMaxD];
    long long tstride[kMaxD];
    const int* start[kMaxD];
    const int* size[kMaxD];
    long long xoff;            // element offset of B / X in the pools
    long long aoff[kMaxD];     // element offset of A_mu / C_mu in the pools
    void* X;                   // block tensor
    void* At[kMaxD];           // coefficient tiles
    void* Ct[kMaxD];
};

// Coefficient tile (I, J), I <= J, of mode mu of equation eq.
struct BatchCoefJob {
    int eq;
    int mu;
    int I;
    int J;
};

struct BatchArgs {
    const WaveArgs* eqs;       // one wavefront parameter block per equation (tiles unused)
    const BatchJob* jobs;      // nullptr: job j is block tiles[j] of equation 0, no count to wait for
    const int* tiles;
    int njobs;
    int* head;                 // next job (zeroed before the launch)
    int* done;                 // finished blocks per equation (zeroed before the launch; may be
                               // nullptr when jobs is)
    int* abort;                // set when any wait ran out of time: later waits give up at once
    long long timeout_ns;
};

// Persistent launch of `grid` CTAs (equations of order d, one form).  prod
// (ProductKind) selects the arithmetic of the block updates: native, or for
// T = float TF32 / BF16 tensor-core products.
template <typename T>
cudaError_t launch_batched(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s, int prod = kProdNative);
template <typename T>
cudaError_t prepare_batched();
// The paper's two-term form Eq. (3.1), FP64, d = 2..4: persistent launch,
// its occupancy and kernel attributes.
cudaError_t launch_batched_tt(int d, const BatchArgs& a, int grid, cudaStream_t s);
int batched_occupancy_tt(int d);
cudaError_t prepare_batched_tt();
// Complex FP64 (complex-triangular coefficients), d = 1..4, Laplace or d-term form.
cudaError_t launch_batched_z(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s);
int batched_occupancy_z(int d, bool gen);
cudaError_t prepare_batched_z();
// The double-float solve (TSYLV_DF64), d = 1..4, Laplace and d-term forms.
cudaError_t launch_batched_df(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s);
int batched_occupancy_df(int d, bool gen);
cudaError_t prepare_batched_df();
// The two-term form Eq. (3.1) in double-float arithmetic, d = 2..4.
cudaError_t launch_batched_tt_df(int d, const BatchArgs& a, int grid, cudaStream_t s);
int batched_occupancy_tt_df(int d);
cudaError_t prepare_batched_tt_df();
// *dst = a, by one thread (a captured launch keeps `a` by value).
cudaError_t launch_store_args(const WaveArgs& a, WaveArgs* dst, cudaStream_t s);
// Resident CTAs per SM of the persistent kernel.
template <typename T>
int batched_occupancy(int d, bool gen, int prod = kProdNative);

// Block tensors of B and coefficient tiles of every equation; back to X.
template <typename T>
cudaError_t launch_batch_pack(const BatchGeom* g, const BatchJob* jobs, int njobs, const BatchCoefJob* cjobs,
                              int ncjobs, const double* B, const double* A, const double* C, cudaStream_t s);
template <typename T>
cudaError_t launch_batch_unpack(const BatchGeom* g, const BatchJob* jobs, int njobs, double* X, cudaStream_t s);
// Sub-diagonals of every A_mu: out[ooff[k] + i] = A_k(i + 1, i), k over all matrices.
cudaError_t launch_batch_subdiag(const long long* aoff, const long long* nmat, const long long* ooff, int nmats,
                                 long long maxn, const double* A, double* out, cudaStream_t s);

// Batched refinement (pools of all equations; tile_eq maps a block to its
// equation, nrm holds 4 doubles per equation: sum r^2, max |r|, sum x^2).
cudaError_t launch_bscale(const double* r, float* r32, const int* tile_eq, const double* nrm, long long n, int td,
                          cudaStream_t s);
cudaError_t launch_bupdate(double* x, const float* d32, const int* tile_eq, const double* nrm, double* xpart,
                           long long ntiles, int td, cudaStream_t s);
cudaError_t launch_breduce(const double* part, const double* xpart, const long long* tile_off, int count, double* nrm,
                           cudaStream_t s);
cudaError_t launch_bnorm2(const double* pool, const long long* off, const long long* nmat, const int* upper, int count,
                          long long nmax, double* out, cudaStream_t s);

}  // namespace tsylv
