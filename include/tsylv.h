/*
 * tsylv.h -- C ABI of the GB300 (sm_103a) solver for triangular tensor
 * Sylvester equations.
 *
 * Operation (Chen & Kressner, "Recursive blocked algorithms for linear
 * systems with Kronecker product structure"):
 *
 *   Laplace-like form, Sec. 2, Eq. (2.2):
 *       X x_1 A_1 + X x_2 A_2 + ... + X x_d A_d = B
 *   d-term generalized form (the K-term equation of the Conclusions with
 *   K = d and mode family {A_mu, C_mu}):
 *       sum_mu  X x_1 C_1 ... x_mu A_mu ... x_d C_d = B
 *
 * where Y = X x_mu M means Y_(mu) = M X_(mu) (Sec. 2), A_mu is upper
 * quasi-triangular (real Schur form: 1x1 and 2x2 diagonal blocks, Sec. 2
 * after Alg. 1) and C_mu is upper triangular.  The solution is unique iff
 * no sum of eigenvalues lambda_1 + ... + lambda_d vanishes (Sec. 2) --
 * respectively iff the generalized operator is nonsingular.
 *
 * Method: the recursive blocked algorithm of Sec. 2.1 (Alg. 2) with merged
 * modes in the base case (Sec. 2.2-2.3, Alg. 3).  Every mode is partitioned
 * into blocks that keep the 2x2 Schur blocks whole (opts->partition); the
 * right-hand-side updates of Eq. (2.3a) become block mode-mu products, and
 * the leaves are solved by a back-substitution in which 2x2 Schur blocks are
 * solved as coupled groups (the diagonal blocks after the perfect shuffle of
 * Sec. 2.3).  By default one persistent launch per solve runs every block as
 * soon as the blocks it reads are solved (opts->schedule = 0); the
 * alternative is one launch per anti-diagonal wavefront.  The launches of a
 * call are captured once in a CUDA graph and replayed.  The mixed-precision
 * solves (TSYLV_FP32_REFINED, and TSYLV_TF32_REFINED / TSYLV_BF16_REFINED
 * with tensor-core block updates) solve in low precision and refine in FP64
 * with a double-float residual; their first two steps run pipelined in one
 * launch when the solve is latency-bound (opts->fuse_step).
 *
 * Layout.  Tensors are dense and column-major with mode 1 fastest -- the
 * index map Eq. (2.1): element (i_1, ..., i_d) (0-based) is at
 * i_1 + n_1*(i_2 + n_2*(i_3 + ...)).  A contiguous C-ordered torch tensor of
 * shape (n_d, ..., n_1) has this layout.  Every coefficient matrix is an
 * n_mu x n_mu column-major (LAPACK) array: M(i, j) at M[i + n_mu*j].
 * Entries of A_mu below the first subdiagonal and of C_mu below the diagonal
 * are never read (treated as zero).  A nonzero A_mu(i+1, i) marks a 2x2
 * block at (i, i+1); two consecutive nonzero subdiagonal entries are an error.
 *
 * Pointers.  `n` and the arrays `A`, `C`, `dA`, `dC` are host arrays; the
 * matrices and tensors they point to live in device memory.  All device memory is owned by the
 * caller.  The solver entry points allocate no device memory: every scratch
 * buffer is carved out of `work`, whose size comes from the matching
 * *_workspace_bytes query (256-byte alignment is required).  In-place use
 * (X == B) is allowed.  (The diagnostic tsylv_selftest_wait_timeout is the
 * documented exception.)
 *
 * Streams.  Work is queued on `stream`.  Each call reads the 2x2 block
 * structure of A back to the host (a short synchronisation on `stream`
 * before the solve) and synchronises `stream` again at the end to read the
 * device status flag, so every call returns with its results complete.
 *
 * Status.  0 on success; -i if the i-th argument (1-based) is invalid, as in
 * LAPACK's info; positive values are numerical or runtime conditions listed
 * below.  No call aborts, traps or throws.
 */
#ifndef TSYLV_H
#define TSYLV_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum tsylv_status {
    TSYLV_OK = 0,
    TSYLV_ESINGULAR = 1,    /* a diagonal group system had a zero or tiny pivot   */
    TSYLV_ENONFINITE = 2,   /* NaN or Inf appeared in the solution                */
    TSYLV_ENOCONV = 3,      /* refinement missed opts->tol within max_refine steps */
    TSYLV_ECUDA = 4,        /* a CUDA runtime call failed                         */
    TSYLV_ETIMEOUT = 5,     /* a bounded device-side wait ran out                 */
    TSYLV_EUNSUPPORTED = 6, /* valid arguments outside what this build supports   */
    TSYLV_ESCRATCH = 7      /* problem too large for tsylv_solve_noalloc's array   */
};

enum tsylv_precision {
    TSYLV_FP64 = 0,          /* plain FP64 solve (FP64 pipes)                       */
    TSYLV_FP32_REFINED = 1,  /* FP32 solves + FP64-accurate residual refinement:
                                X_0 = 0; D_k = solve_FP32(R_k / max|R_k|);
                                X_{k+1} = X_k + max|R_k| D_k (FP64);
                                R_{k+1} = B - A(X_{k+1}) (opts->residual)
                                until ||R|| / (||A|| ||X||) <= opts->tol        */
    TSYLV_TF32_REFINED = 2,  /* as TSYLV_FP32_REFINED, with the block updates of the
                                low-precision solve on the tensor cores: operands
                                rounded to TF32, FP32 accumulation (warp-level
                                mma.sync); the in-block back-substitution stays
                                FP32, the residual and X FP64-accurate.  The less
                                accurate correction takes about one refinement
                                step more than TSYLV_FP32_REFINED.  Persistent
                                schedule only (opts->schedule = 1 returns
                                TSYLV_EUNSUPPORTED)                                */
    TSYLV_BF16_REFINED = 3,  /* as TSYLV_TF32_REFINED with BF16 operands (about
                                two steps more than TSYLV_FP32_REFINED)          */
    TSYLV_DF64 = 4           /* one solve in double-float arithmetic on the FP32
                                pipes: every value a pair of floats (about 48
                                significant bits; exact products by FMA, two-sum
                                accumulation), the same partition, schedule and
                                back-substitution as TSYLV_FP64.  No residual is
                                evaluated (info->resid = -1; tsylv_residual
                                measures it).  tsylv_solve / gtsylv_solve, the
                                transposed solves, solve plans,
                                tsylv_solve_batched (d = 1..4) and gsylvten_solve
                                (d = 2..4), persistent schedule; elsewhere
                                TSYLV_EUNSUPPORTED                                 */
};

enum tsylv_residual_kind {
    TSYLV_RESID_DF64 = 0,    /* residual in double-FP32 (~2^-48) arithmetic        */
    TSYLV_RESID_FP64 = 1     /* residual on the native FP64 pipes                   */
};

typedef struct tsylv_opts {
    int precision;    /* enum tsylv_precision, default TSYLV_FP64                    */
    int max_refine;   /* refinement steps for *_REFINED (default 10)                 */
    double tol;       /* target ||B - A(X)|| / (||A|| ||X||) (default 1e-12)         */
    int residual;     /* enum tsylv_residual_kind, default TSYLV_RESID_DF64          */
    int nmin;         /* recursion cutoff: the largest block extent per mode (leaf
                         bound of the split tree).  0 (default): the tile extent
                         TE of the order d (32, 16, 8, 4, 4 for d = 1..5); 2..TE: that
                         bound for every mode; -1: autotuned.  A single solve tunes
                         on its first call per order, mode sizes, form, direction
                         and precision (each candidate tile shape -- every mode TE,
                         TE - 1, 3/4 TE or TE/2, or TE/2 in the last mode only
                         -- solves once, timed; X is written, B is not; an
                         in-place call takes the default).  tsylv_solve_batched
                         tunes by default (0 or -1) together with its launch.
                         Values above TE, and 1, return TSYLV_EUNSUPPORTED.       */
    int split;        /* largest cluster size for split block updates; 0 = auto      */
    int use_graph;    /* 1 (default): capture each schedule once and replay it      */
    int host_io;      /* reserved (host-resident operands); must be 0: this build
                         returns TSYLV_EUNSUPPORTED otherwise                        */
    int timing;       /* 1: time the phases with CUDA events (fields t_* of info)    */
    int schedule;     /* block schedule of a solve: 0 (default) one persistent
                         dataflow launch (a block starts as soon as each source
                         block it reads is solved); 1 one launch per anti-diagonal
                         wavefront (split over a cluster when the wavefront is short) */
    int partition;    /* blocks of each mode: 0 (default) tile-aligned blocks of the
                         largest extent, a boundary moved back by one where it
                         would cut a 2x2 block; 1 the leaves of the halving split
                         rule of Alg. 2.  Both give the same solution up to rounding. */
    int resid_update; /* *_REFINED: 0 (default) from the second refinement step on,
                         once the relative residual is <= 1e-5, the residual is
                         updated from the step's FP32 correction, R -= s A(D) in
                         FP32 (error ~2^-24 |A| |s D|, far below the residual);
                         1: the full FP64-accurate residual at every step         */
    int fuse_step;    /* *_REFINED, Laplace form, d >= 2, DF64 residual, schedule 0:
                         2 runs the first two steps as one launch, the second
                         solve and both residuals following the first solve block
                         by block (the same result as separate steps, bit for
                         bit); 3 separate launches; 0 (default) 2 when the
                         solve's largest wavefront has fewer blocks than the GPU
                         has resident CTAs for it (latency-bound), 3 otherwise.
                         Other forms: separate.  1 (the first step alone in one
                         launch) is no longer offered: TSYLV_EUNSUPPORTED       */
    int wait_ms;      /* bound of every device-side wait (a source block's "solved"
                         flag, a bulk copy), in milliseconds: 1 .. 600000, default
                         2000.  A wait that runs out ends the launch and the call
                         returns TSYLV_ETIMEOUT; raise it on a GPU shared with
                         long-running work                                        */
    int leaf[5];      /* per-mode leaf bounds (tile shape), overriding nmin mode by
                         mode: entry mu in 2..TE bounds the blocks of mode mu, 0
                         takes nmin's bound (TE when nmin <= 0).  Any nonzero entry
                         fixes the shape (no autotuning).  Default all 0.         */
    int fp64_update;  /* arithmetic of the block updates of a TSYLV_FP64 solve
                         (ignored by the refined precisions): 0 (default) and 1
                         FP64 fused multiply-adds; 2 FP64 DMMA tensor-core
                         instructions (mma m8n8k4, FP64 accumulation), built for
                         tsylv_solve / gtsylv_solve (and the transposed solves)
                         at d = 2, 3 on the persistent schedule -- elsewhere
                         TSYLV_EUNSUPPORTED.  DMMA and FMA share the FP64 units of
                         this GPU; DMMA measured 0-18% slower, hence not the
                         default.  Both skip the zero padding of short blocks;
                         results agree to rounding.                              */
} tsylv_opts;

typedef struct tsylv_info {
    int iterations;       /* refinement steps taken (0 for TSYLV_FP64)              */
    int waves;            /* wavefront launches per solve                           */
    int launches;         /* kernels launched by the call                           */
    int tiles;            /* blocks of the block grid                               */
    double resid;         /* final ||B - A(X)|| / (||A|| ||X||) when computed, else -1 */
    double norm_A;        /* the ||A|| used above (sum_mu ||A_mu||_2 prod ||C_eta||_2) */
    double flops;         /* floating-point operations executed per solve           */
    double t_total_ms;    /* opts->timing: device time of the whole call             */
    double t_waves_ms;    /* opts->timing: device time of the wavefront launches     */
    double t_resid_ms;    /* opts->timing: device time of the residual launches      */
    int batch_order;      /* tsylv_solve_batched: job-queue order used (0 longest remaining
                             path first, 1 wavefront-major, 2 equation-major)      */
    int batch_ctas_per_sm;/* tsylv_solve_batched: resident CTAs per SM used          */
    int leaf[5];          /* leaf bound (recursion cutoff) of every mode in the block
                             partition used -- the tile shape (opts->nmin); for a
                             batch, that of its equations of the highest order d   */
} tsylv_info;

/* Fill *opts with the defaults listed above. */
void tsylv_opts_default(tsylv_opts* opts);

/* Human-readable text of a status code (static storage). */
const char* tsylv_status_string(int status);

/* Text of the last CUDA runtime failure seen by a call of this thread
 * (TSYLV_ECUDA), naming the failing step; "" if none.  Valid until the next
 * call on the same thread. */
const char* tsylv_last_error(void);

/* Workspace bytes for tsylv_solve (generalized = 0) / gtsylv_solve
 * (generalized = 1) and their transposed variants.  Returns 0 for invalid
 * arguments.  d in 1..5 (1..4 for the generalized form), every n[mu] >= 1. */
size_t tsylv_workspace_bytes(int d, const int64_t* n, int generalized, const tsylv_opts* opts);

/* Solve the Laplace-like equation Eq. (2.2).
 *   d          number of modes (1..5)
 *   n          host array of d mode sizes
 *   A          host array of d pointers to the n_mu x n_mu upper
 *              quasi-triangular coefficients
 *   B          right-hand side tensor (read only)
 *   X          solution tensor (written; may equal B)
 *   work       device workspace of work_bytes >= tsylv_workspace_bytes(...)
 *   opts       NULL for the defaults
 *   info       optional output (may be NULL)
 *   stream     CUDA stream (0 = legacy default stream)
 * Errors: -1..-10 for the corresponding argument; TSYLV_ESINGULAR when a
 * group pivot of the back-substitution is zero or below 16 eps times the
 * group's largest entry; TSYLV_ENONFINITE for NaN/Inf in X; TSYLV_ENOCONV for
 * a refined solve that missed opts->tol (X then holds the last iterate). */
int tsylv_solve(int d, const int64_t* n, const double* const* A, const double* B, double* X,
                void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                cudaStream_t stream);

/* Solve the d-term generalized equation sum_mu X x_mu A_mu x_{eta!=mu} C_eta = B.
 * C: host array of d pointers to the upper triangular C_mu.  Other arguments
 * and errors as tsylv_solve (argument numbers shift by one after A). */
int gtsylv_solve(int d, const int64_t* n, const double* const* A, const double* const* C,
                 const double* B, double* X, void* work, size_t work_bytes,
                 const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);

/* Transposed equations A^T(L) = G: the coefficients enter as A_mu^T (lower
 * quasi-triangular) and C_mu^T.  Solved by the index flip J A_mu^T J (J the
 * reversal permutation), which is upper quasi-triangular again, so the same
 * recursion runs in reversed order.  Arguments as the forward calls
 * (B -> G, X -> L). */
int tsylv_solve_transposed(int d, const int64_t* n, const double* const* A, const double* G,
                           double* L, void* work, size_t work_bytes, const tsylv_opts* opts,
                           tsylv_info* info, cudaStream_t stream);
int gtsylv_solve_transposed(int d, const int64_t* n, const double* const* A,
                            const double* const* C, const double* G, double* L, void* work,
                            size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                            cudaStream_t stream);

/* Solve plans: repeated FP64 solves of Eq. (2.2) or of the d-term form (forward
 * or transposed) with the same mode sizes, the same coefficient pointers and
 * the same 2x2 block structure of the A_mu, queued without host
 * synchronisation.  tsylv_solve synchronises its stream twice per call (it
 * reads the 2x2 structure back to plan the block partition, and reads the
 * status word); a plan reads the structure once, at creation, and an
 * execution only enqueues work, so a caller can queue solves back to back and
 * overlap them with its own copies and kernels.
 *
 * tsylv_plan_create: d, n, A, C (NULL: the Laplace form), transposed (0 / 1),
 *   work / work_bytes (the workspace of tsylv_workspace_bytes(d, n, C != NULL,
 *   opts); it only has to be valid during the call and during executions),
 *   opts (TSYLV_FP64 or TSYLV_DF64; nmin >= 0 or leaf bounds -- no
 *   autotuning; no event timing; fp64_update as for tsylv_solve).  Reads the structure (one
 *   synchronisation of `stream`), builds the partition and schedule, and keeps
 *   a copy of the structure on the device (one byte per subdiagonal entry,
 *   allocated here).  Returns 0 and sets *plan, -i for a bad i-th argument
 *   (-4: A violates the quasi-triangular structure), TSYLV_EUNSUPPORTED or
 *   TSYLV_ECUDA.
 * tsylv_plan_execute: enqueues one whole solve on `stream` -- coefficient
 *   tiles packed from the plan's A_mu (C_mu) pointers, whose VALUES may change
 *   between executions, right-hand side packed from B, the persistent solve,
 *   the unpack into X -- and returns without waiting.  If status is not NULL
 *   (a device int), the execution writes its TSYLV status code there when the
 *   stream reaches it: 0, 1 singular, 2 non-finite, 5 wait timed out, 4 device
 *   self-check, -3 the A_mu no longer have the plan's 2x2 structure (checked
 *   on the device at every execution; the solution is then meaningless).  The
 *   return value only reports the enqueue: 0, -1 null plan, -2 null B, -3 null
 *   X, -4 work not 256-byte aligned, -5 work_bytes too small,
 *   TSYLV_EUNSUPPORTED on another device than the plan's, TSYLV_ECUDA.
 *   Executions sharing a workspace must be ordered (one stream, or events):
 *   the workspace holds the block tensors of the solve in flight.  The first
 *   execution for a given (B, X, work) builds a CUDA graph (host work only).
 * tsylv_plan_destroy: frees the plan (after the last execution has finished:
 *   it synchronises the device). */
typedef struct tsylv_plan_s* tsylv_plan;
int tsylv_plan_create(tsylv_plan* plan, int d, const int64_t* n, const double* const* A, const double* const* C,
                      int transposed, void* work, size_t work_bytes, const tsylv_opts* opts, cudaStream_t stream);
int tsylv_plan_execute(tsylv_plan plan, const double* B, double* X, void* work, size_t work_bytes, int* status,
                       cudaStream_t stream);
void tsylv_plan_destroy(tsylv_plan plan);

/* The complex-triangular variant (Sec. 2.4: the paper's experiments reduce
 * every coefficient to complex Schur form, which is upper triangular): the
 * Laplace form Eq. (2.2) (ztsylv_solve) or the d-term generalized form
 * (zgtsylv_solve) with complex FP64 coefficients, right-hand side and
 * solution.  Every complex array is interleaved (re, im) pairs of doubles --
 * C99 double complex, std::complex<double>, torch.complex128 -- in the
 * layouts of tsylv_solve (tensors column-major, matrices column-major
 * n_mu x n_mu); the pointers are passed as double*.  A_mu and C_mu are upper
 * triangular: entries below the diagonal are never read (no 2x2 blocks).  The
 * same block partition, persistent schedule and back-substitution as the real
 * solves, in complex arithmetic (a complex multiply-add is four real FP64
 * fused multiply-adds; the reciprocal of a diagonal entry uses Smith's
 * quotient).  d = 1..4; FP64 only (other precisions, opts->schedule = 1 and
 * nmin = -1 return TSYLV_EUNSUPPORTED); arguments and statuses as
 * tsylv_solve / gtsylv_solve.  work: ztsylv_workspace_bytes(d, n, generalized, opts). */
size_t ztsylv_workspace_bytes(int d, const int64_t* n, int generalized, const tsylv_opts* opts);
int ztsylv_solve(int d, const int64_t* n, const double* const* A, const double* B, double* X, void* work,
                 size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);
int zgtsylv_solve(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                  double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                  cudaStream_t stream);

/* The paper's own generalized form, Sec. 3, Eq. (3.1):
 *       X x_1 A_1 + X x_1 C x_2 A_2 x_3 ... x_d A_d = B,
 * i.e. (I x ... x I x A_1 + A_d x ... x A_2 x C) vec(X) = vec(B) (Eq. (1.5)),
 * with every A_mu upper quasi-triangular and C upper triangular (the form
 * Alg. 4 reduces general coefficients to).  With A_1 = -lambda I it is the
 * shifted Kronecker system of Eq. (1.6).  Solved by the recursion of
 * Sec. 3.1 (Alg. 5; the merged base case of Alg. 6 solved directly): the
 * same block partition and persistent schedule as tsylv_solve, the block
 * updates being the A_1 term along mode 1 and the chain
 * Q_l = X x_l A_l ... x_d A_d carried per block (Horner order over the modes,
 * C in mode 1); 2x2 blocks of any A_mu are solved as coupled groups.
 *   d      2..4 (1 and 5 return TSYLV_EUNSUPPORTED)
 *   A      host array of d device pointers: A_1 .. A_d, n_mu x n_mu
 *   C      device pointer: the n_1 x n_1 upper triangular C
 *   B, X   as tsylv_solve (X may equal B); work of gsylvten_workspace_bytes
 * Options: precision TSYLV_FP64 or TSYLV_DF64 (other precisions,
 * opts->schedule = 1, fp64_update = 2 and autotuning nmin = -1 return
 * TSYLV_EUNSUPPORTED); nmin >= 2, leaf, split, partition,
 * use_graph, timing, wait_ms as for tsylv_solve.  Arguments: 1 d, 2 n, 3 A,
 * 4 C, 5 B, 6 X, 7 work, 8 work_bytes, 9 opts; statuses as tsylv_solve. */
size_t gsylvten_workspace_bytes(int d, const int64_t* n, const tsylv_opts* opts);
int gsylvten_solve(int d, const int64_t* n, const double* const* A, const double* C, const double* B,
                   double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                   cudaStream_t stream);

/* Workspace bytes for tsylv_residual. */
size_t tsylv_residual_workspace_bytes(int d, const int64_t* n, int generalized);

/* Residual R = B - A(X) (C == NULL: Laplace form) with the arithmetic chosen
 * by opts->residual: TSYLV_RESID_FP64 multiplies and adds on the FP64 pipes;
 * TSYLV_RESID_DF64 carries every double as an unevaluated pair of floats
 * (error <= 2^-48 relative per entry) and runs on the FP32 pipes.  *rel
 * (optional, host) receives ||R||_F / (||A|| ||X||_F) with
 * ||A|| = sum_mu ||A_mu||_2 prod_{eta!=mu} ||C_eta||_2 (power-iteration
 * estimates of the 2-norms).  Arguments: 1 d, 2 n, 3 A, 4 C, 5 B, 6 X, 7 R,
 * 8 rel, 9 work, 10 work_bytes (>= tsylv_residual_workspace_bytes), 11 opts,
 * 12 stream. */
int tsylv_residual(int d, const int64_t* n, const double* const* A, const double* const* C,
                   const double* B, const double* X, double* R, double* rel, void* work,
                   size_t work_bytes, const tsylv_opts* opts, cudaStream_t stream);

/* Workspace bytes for tsylv_backward. */
size_t tsylv_backward_workspace_bytes(int d, const int64_t* n, int generalized,
                                      const tsylv_opts* opts);

/* Adjoint of X = A^{-1}(B) for a scalar loss with gradient dX = dL/dX:
 *   Lambda = A^{-T}(dX)                                 (transposed solve)
 *   dB     = Lambda
 *   dA_mu  = -mask_A( Lambda_(mu) [X x_{eta!=mu} C_eta]_(mu)^T )
 *   dC_mu  = -mask_C( sum_{nu!=mu} Lambda_(mu) [X x_nu A_nu x_{eta!=mu,nu} C_eta]_(mu)^T )
 * mask_A keeps the upper triangle and the subdiagonal entries of the 2x2
 * blocks of A_mu; mask_C keeps the upper triangle.  C == NULL: Laplace form
 * (then dC is ignored).  dB may be NULL; dA, dC may be NULL or hold NULL
 * entries for gradients that are not wanted.  X is the forward solution. */
int tsylv_backward(int d, const int64_t* n, const double* const* A, const double* const* C,
                   const double* X, const double* dX, double* dB, double* const* dA,
                   double* const* dC, void* work, size_t work_bytes, const tsylv_opts* opts,
                   tsylv_info* info, cudaStream_t stream);

/* Workspace bytes for tsylv_solve_batched. */
size_t tsylv_batched_workspace_bytes(int count, const int* d, const int64_t* n_packed,
                                     int generalized, const tsylv_opts* opts);

/* Many independent equations of different sizes in one persistent launch
 * (per order d present in the batch), captured with the packing and
 * unpacking in one CUDA graph when opts->use_graph.  Each equation is solved
 * exactly as tsylv_solve / gtsylv_solve would solve it (same block partition
 * from the split rule of Alg. 2, same block updates and base case), so every
 * result equals the corresponding single solve up to rounding.
 *   count       number of equations (>= 1)
 *   d           host array [count] of orders (1..5; 1..4 with C_pool)
 *   n_packed    host array: the mode sizes of all equations, concatenated
 *   off_A       host array [sum d]: element offset of each A_mu (and C_mu) in
 *               A_pool / C_pool, in the order of n_packed; every matrix is
 *               column-major n_mu x n_mu
 *   off_X       host array [count]: element offset of each tensor in B_pool /
 *               X_pool (column-major, mode 1 fastest)
 *   A_pool, C_pool, B_pool, X_pool   device pools; C_pool NULL for the
 *               Laplace form (all equations share one form); X_pool may equal
 *               B_pool
 *   work        device workspace of tsylv_batched_workspace_bytes bytes,
 *               256-byte aligned, caller-owned
 * Precision: TSYLV_FP64; TSYLV_DF64 (the double-float solve, every order
 * d <= 4); or TSYLV_FP32_REFINED when every equation of the batch has the same
 * order d (FP32 solves of all equations in one persistent launch, FP64
 * residuals and corrections per equation, each equation refined to
 * opts->tol); other values return TSYLV_EUNSUPPORTED.
 * Launch parameters: on the first call for a given set of shapes and 2x2
 * structures a built-in autotuner times the job-queue orders (longest
 * remaining path first, wavefront-major, equation-major) and the resident
 * CTAs per SM on this batch and keeps the fastest (info->batch_order,
 * info->batch_ctas_per_sm); opts->split > 0 fixes the CTAs per SM instead.
 * The block extent (the recursion cutoff) is that of a single solve.
 * Errors: -i for a bad i-th argument (-6 when some A_mu is not quasi-
 * triangular); numerical statuses as for tsylv_solve, combined (the first
 * nonzero in equation order wins); per_status (optional, host [count])
 * receives each equation's own.  Synchronises the stream before returning. */
int tsylv_solve_batched(int count, const int* d, const int64_t* n_packed, const int64_t* off_A,
                        const int64_t* off_X, const double* A_pool, const double* C_pool,
                        const double* B_pool, double* X_pool, void* work, size_t work_bytes,
                        const tsylv_opts* opts, int* per_status, tsylv_info* info,
                        cudaStream_t stream);

/* Allocation-free variant of tsylv_solve (FP64 precision only).  The paper
 * has no counterpart: this entry point serves callers that cannot allocate
 * device memory when they solve -- a host application whose own allocator owns
 * all device memory, a real-time loop that cannot afford cudaMalloc's latency
 * and implicit synchronisation, a plug-in that may not grow the process's
 * device footprint after start-up.  The caller passes A, B and X as for
 * tsylv_solve; there is no workspace argument.  All scratch lives in one
 * file-scope device array of 32 MiB, which every GPU that loads the library
 * holds until the process exits; problems whose workspace (the
 * tsylv_workspace_bytes bound) exceeds it are rejected with TSYLV_ESCRATCH and
 * a tsylv_last_error() message, before any GPU work.  The first call on each
 * device looks up the array's device address and sets kernel attributes; make
 * that first call before any stream capture.  Like tsylv_solve, every call
 * synchronises `stream` twice: after reading back the 2x2 structure of A and
 * at the end, to read the status.  Calls share the array, so calls whose GPU
 * work overlaps race on it: serialise them.  The status word is cleared by
 * every call.  Arguments and status codes as tsylv_solve, with opts the 6th
 * argument: its fields are checked as tsylv_solve checks them (-6 for a field
 * out of range, TSYLV_EUNSUPPORTED for host_io or an nmin outside 0, 2..TE);
 * opts->precision must be TSYLV_FP64 (else -6), opts->timing 0,
 * opts->nmin not -1 (no autotuning runs) and opts->fp64_update not 2 (its
 * block updates are FP64 FMA); else TSYLV_EUNSUPPORTED.  The schedule is always one launch per anti-diagonal
 * wavefront (opts->schedule is not used). */
int tsylv_solve_noalloc(int d, const int64_t* n, const double* const* A, const double* B, double* X,
                        const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream);

/* Change of basis of a tensor (Alg. 1: right-hand side in, solution out; Sec. 3's generalized
 * Schur factors Q, Z for the d-term form): Y = X x_1 op(M_1) x_2 op(M_2) ...
 * x_d op(M_d), with op(M) = M (trans[mu] == 0) or M^T (trans[mu] != 0; trans
 * may be NULL: no transposes) and X x_mu N the mode-mu product
 * (Y(.., i, ..) = sum_k N(i, k) X(.., k, ..)).  M[mu] == NULL skips mode mu.
 * With orthogonal Schur factors this takes an equation with general
 * coefficients to the quasi-triangular form tsylv_solve / gtsylv_solve take
 * (B x_mu U_mu^T), and the solution back (X x_mu U_mu).  Dense FP64 matrix
 * products on the FP64 tensor cores (the library's own DMMA kernel, one launch
 * per transformed mode, on `stream`).  X, Y: column-major device tensors, Y may equal X;
 * M[mu]: column-major n_mu x n_mu device matrices.  work: device memory of at
 * least tsylv_transform_workspace_bytes(d, n) bytes, 256-byte aligned.
 * Returns 0, -i for a bad i-th argument (before any GPU work), or TSYLV_ECUDA. */
size_t tsylv_transform_workspace_bytes(int d, const int64_t* n);
int tsylv_transform(int d, const int64_t* n, const double* const* M, const int* trans, const double* X, double* Y,
                    void* work, size_t work_bytes, cudaStream_t stream);

/* Diagnostic of the failure path of the persistent schedule (every inter-block
 * wait of a solve is bounded): runs the dataflow launch of a small FP64 solve
 * (d = 2, 32 x 32, 2 x 2 blocks) with its first block withheld from the job
 * queue, so that the blocks reading it wait for a "solved" flag that nothing
 * sets.  The wait runs out after timeout_ns (1 ms .. 10 s), raises the
 * launch-wide abort word, every other wait gives up at once, the kernel ends
 * and the status word is read back: the call returns TSYLV_ETIMEOUT when this
 * path works (TSYLV_ECUDA, or another code, otherwise), and the CUDA context
 * stays usable.  It allocates and frees its own device memory (cudaMalloc /
 * cudaFree) and synchronises `stream`.  Not a solver entry point. */
int tsylv_selftest_wait_timeout(long long timeout_ns, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSYLV_H */
