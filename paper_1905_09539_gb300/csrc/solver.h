// Solver entry points behind the C ABI.
#pragma once

#include <vector>

#include "tsylv_internal.h"

namespace tsylv {

size_t solver_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o, bool transposed);
int solver_solve(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
                 void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream,
                 bool gen, bool transposed);
size_t solver_residual_workspace_bytes(int d, const int64_t* n, bool gen);
int solver_selftest_wait_timeout(long long timeout_ns, cudaStream_t stream);
size_t transform_workspace_bytes(int d, const int64_t* n);
int transform(int d, const int64_t* n, const double* const* M, const int* trans, const double* X, double* Y,
              void* work, size_t work_bytes, cudaStream_t stream);
int solver_residual(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                    const double* X, double* R, double* rel, void* work, size_t work_bytes, const tsylv_opts* opts,
                    cudaStream_t stream);
size_t solver_backward_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o);
int solver_backward(int d, const int64_t* n, const double* const* A, const double* const* C, const double* X,
                    const double* dX, double* dB, double* const* dA, double* const* dC, void* work, size_t work_bytes,
                    const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);
size_t solver_batched_workspace_bytes(int count, const int* d, const int64_t* n_packed, bool gen, const tsylv_opts& o);
int solver_batched(int count, const int* d, const int64_t* n_packed, const int64_t* off_A, const int64_t* off_X,
                   const double* A_pool, const double* C_pool, const double* B_pool, double* X_pool, void* work,
                   size_t work_bytes, const tsylv_opts* opts, int* per_status, tsylv_info* info, cudaStream_t stream);

cudaStream_t capture_stream();

// Solve plans (tsylv_plan_*): opaque handles of repeated FP64 solves.
int plan_create(void** out, int d, const int64_t* n, const double* const* A, const double* const* C, bool flip,
                void* work, size_t work_bytes, const tsylv_opts* opts, cudaStream_t stream);
int plan_execute(void* handle, const double* B, double* X, void* work, size_t work_bytes, int* status,
                 cudaStream_t stream);
void plan_destroy(void* handle);

size_t solver_tt_workspace_bytes(int d, const int64_t* n, const tsylv_opts& o);
size_t solver_z_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o);
int solver_solve_z(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                   double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                   cudaStream_t stream, bool gen);
int solver_solve_tt(int d, const int64_t* n, const double* const* A, const double* Cm, const double* B, double* X,
                    void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);

// Tile shape of opts->nmin: 0 the default, nmin > 0 that uniform leaf bound,
// -1 (autotuned) any candidate.
int shape_of_nmin(int nmin);
// Tile shape of the options: opts->leaf (per-mode bounds, zero entries take
// nmin's) when any entry is set, else shape_of_nmin.
int shape_of_opts(const tsylv_opts& o, int d);

// Shared argument checks of the solve entry points.
bool solve_shape_ok(int d, const int64_t* n);
// 0, -1 for an option field out of its range, or TSYLV_EUNSUPPORTED for a
// valid request this build does not serve (host_io, nmin 1 or above the tile
// extent, fuse_step 1).
int check_opts(const tsylv_opts& o, int d);
// 2x2 block structure of every A_mu: the sub-diagonal is gathered into
// base + 256, read back (a synchronisation of `stream`) and validated (-3
// for two adjacent 2x2 blocks); flipped for the transposed equation.
int solve_read_structure(int d, const long long* n, const double* const* A, char* base, bool flip,
                         cudaStream_t stream, std::vector<uint8_t>& sub);

int solver_solve_noalloc(int d, const int64_t* n, const double* const* A, const double* B, double* X,
                         const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);

}  // namespace tsylv
