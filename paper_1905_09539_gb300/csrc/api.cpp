// C ABI entry points (include/tsylv.h): argument checks, structure read-back,
// schedule lookup, CUDA-graph capture/replay and status read-back.
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "plan.h"
#include "solver.h"

using namespace tsylv;

namespace {
thread_local std::string g_last_error;
}

namespace tsylv {
int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return TSYLV_ECUDA;
}
int cuda_fail_msg(const char* where) {
    g_last_error = where;
    return TSYLV_ECUDA;
}
}  // namespace tsylv

extern "C" const char* tsylv_last_error(void) { return g_last_error.c_str(); }

extern "C" void tsylv_opts_default(tsylv_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = TSYLV_FP64;
    o->max_refine = 10;
    o->tol = 1e-12;
    o->residual = TSYLV_RESID_DF64;
    o->nmin = 0;
    o->split = 0;
    o->use_graph = 1;
    o->host_io = 0;
    o->timing = 0;
    o->schedule = 0;
    o->partition = 0;
    o->resid_update = 0;
    o->fuse_step = 0;
    o->wait_ms = 2000;
}

extern "C" const char* tsylv_status_string(int s) {
    if (s < 0) return "invalid argument (-i: the i-th argument)";
    switch (s) {
        case TSYLV_OK: return "ok";
        case TSYLV_ESINGULAR: return "singular diagonal group system";
        case TSYLV_ENONFINITE: return "non-finite value in the solution";
        case TSYLV_ENOCONV: return "refinement did not reach the tolerance";
        case TSYLV_ECUDA: return "CUDA runtime error";
        case TSYLV_ETIMEOUT: return "bounded device wait timed out";
        case TSYLV_EUNSUPPORTED: return "unsupported configuration";
        case TSYLV_ESCRATCH: return "problem exceeds the static scratch of tsylv_solve_noalloc";
        default: return "unknown status";
    }
}

extern "C" size_t tsylv_workspace_bytes(int d, const int64_t* n, int generalized, const tsylv_opts* opts) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    return solver_workspace_bytes(d, n, generalized != 0, o, false);
}

extern "C" int tsylv_solve(int d, const int64_t* n, const double* const* A, const double* B, double* X, void* work,
                           size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    return solver_solve(d, n, A, nullptr, B, X, work, work_bytes, opts, info, stream, false, false);
}

extern "C" int gtsylv_solve(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                            double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                            cudaStream_t stream) {
    return solver_solve(d, n, A, C, B, X, work, work_bytes, opts, info, stream, true, false);
}

extern "C" int tsylv_solve_transposed(int d, const int64_t* n, const double* const* A, const double* G, double* L,
                                      void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                                      cudaStream_t stream) {
    return solver_solve(d, n, A, nullptr, G, L, work, work_bytes, opts, info, stream, false, true);
}

extern "C" int gtsylv_solve_transposed(int d, const int64_t* n, const double* const* A, const double* const* C,
                                       const double* G, double* L, void* work, size_t work_bytes,
                                       const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    return solver_solve(d, n, A, C, G, L, work, work_bytes, opts, info, stream, true, true);
}

extern "C" int tsylv_plan_create(tsylv_plan* plan, int d, const int64_t* n, const double* const* A,
                                 const double* const* C, int transposed, void* work, size_t work_bytes,
                                 const tsylv_opts* opts, cudaStream_t stream) {
    if (!plan) return -1;
    if (transposed != 0 && transposed != 1) return -6;
    void* h = nullptr;
    const int st = plan_create(&h, d, n, A, C, transposed != 0, work, work_bytes, opts, stream);
    *plan = static_cast<tsylv_plan>(h);
    return st;
}

extern "C" int tsylv_plan_execute(tsylv_plan plan, const double* B, double* X, void* work, size_t work_bytes,
                                  int* status, cudaStream_t stream) {
    return plan_execute(plan, B, X, work, work_bytes, status, stream);
}

extern "C" void tsylv_plan_destroy(tsylv_plan plan) { plan_destroy(plan); }

extern "C" size_t ztsylv_workspace_bytes(int d, const int64_t* n, int generalized, const tsylv_opts* opts) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    return solver_z_workspace_bytes(d, n, generalized != 0, o);
}

extern "C" int ztsylv_solve(int d, const int64_t* n, const double* const* A, const double* B, double* X, void* work,
                            size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    return solver_solve_z(d, n, A, nullptr, B, X, work, work_bytes, opts, info, stream, false);
}

extern "C" int zgtsylv_solve(int d, const int64_t* n, const double* const* A, const double* const* C,
                             const double* B, double* X, void* work, size_t work_bytes, const tsylv_opts* opts,
                             tsylv_info* info, cudaStream_t stream) {
    return solver_solve_z(d, n, A, C, B, X, work, work_bytes, opts, info, stream, true);
}

extern "C" size_t gsylvten_workspace_bytes(int d, const int64_t* n, const tsylv_opts* opts) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    return solver_tt_workspace_bytes(d, n, o);
}

extern "C" int gsylvten_solve(int d, const int64_t* n, const double* const* A, const double* C, const double* B,
                              double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                              cudaStream_t stream) {
    return solver_solve_tt(d, n, A, C, B, X, work, work_bytes, opts, info, stream);
}

extern "C" size_t tsylv_transform_workspace_bytes(int d, const int64_t* n) { return transform_workspace_bytes(d, n); }

extern "C" int tsylv_transform(int d, const int64_t* n, const double* const* M, const int* trans, const double* X,
                               double* Y, void* work, size_t work_bytes, cudaStream_t stream) {
    return transform(d, n, M, trans, X, Y, work, work_bytes, stream);
}

extern "C" int tsylv_selftest_wait_timeout(long long timeout_ns, cudaStream_t stream) {
    return solver_selftest_wait_timeout(timeout_ns, stream);
}

extern "C" size_t tsylv_residual_workspace_bytes(int d, const int64_t* n, int generalized) {
    return solver_residual_workspace_bytes(d, n, generalized != 0);
}

extern "C" int tsylv_residual(int d, const int64_t* n, const double* const* A, const double* const* C,
                              const double* B, const double* X, double* R, double* rel, void* work, size_t work_bytes,
                              const tsylv_opts* opts, cudaStream_t stream) {
    return solver_residual(d, n, A, C, B, X, R, rel, work, work_bytes, opts, stream);
}

extern "C" size_t tsylv_backward_workspace_bytes(int d, const int64_t* n, int generalized, const tsylv_opts* opts) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    return solver_backward_workspace_bytes(d, n, generalized != 0, o);
}

extern "C" int tsylv_backward(int d, const int64_t* n, const double* const* A, const double* const* C, const double* X,
                              const double* dX, double* dB, double* const* dA, double* const* dC, void* work,
                              size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    return solver_backward(d, n, A, C, X, dX, dB, dA, dC, work, work_bytes, opts, info, stream);
}

extern "C" size_t tsylv_batched_workspace_bytes(int count, const int* d, const int64_t* n_packed, int generalized,
                                                const tsylv_opts* opts) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    return solver_batched_workspace_bytes(count, d, n_packed, generalized != 0, o);
}

extern "C" int tsylv_solve_batched(int count, const int* d, const int64_t* n_packed, const int64_t* off_A,
                                   const int64_t* off_X, const double* A_pool, const double* C_pool,
                                   const double* B_pool, double* X_pool, void* work, size_t work_bytes,
                                   const tsylv_opts* opts, int* per_status, tsylv_info* info, cudaStream_t stream) {
    return solver_batched(count, d, n_packed, off_A, off_X, A_pool, C_pool, B_pool, X_pool, work, work_bytes, opts,
                          per_status, info, stream);
}
