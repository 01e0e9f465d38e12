// Internal declarations shared by the host schedule code and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/tsylv.h"
#include "complex_z.h"
#include "double_float.h"

namespace tsylv {

constexpr int kMaxD = 5;
constexpr int kThreads = 128;       // threads per CTA of the block kernels
constexpr int kMaxCluster = 8;      // portable cluster size for split block updates

// Block extent per mode (the leaf size n_min of the split tree) as a function
// of the order d: the block holds at most 512 unknowns (1024 for d = 5).
__host__ __device__ constexpr int tile_extent(int d) { return d == 1 ? 32 : d == 2 ? 16 : d == 3 ? 8 : 4; }
__host__ __device__ constexpr int ipow(int b, int e) {
    int r = 1;
    for (int i = 0; i < e; i++) r *= b;
    return r;
}

// Row (mode-MU index) of in-block element e = threadIdx.x + q * kThreads for a
// mode of stride st: when st * TE divides kThreads it is the same for every
// slot q of the thread, and is written so, so that the loads of a coefficient
// row are shared by the thread's slots.
#if defined(__CUDACC__)
template <int TE, int st>
__device__ __forceinline__ int row_of(int e) {
    if constexpr (kThreads % (st * TE) == 0) return (static_cast<int>(threadIdx.x) / st) % TE;
    else return (e / st) % TE;
}
#endif

// Record a CUDA failure for tsylv_last_error(); returns TSYLV_ECUDA.
int cuda_fail(cudaError_t e, const char* where);
// Same for a failure with no CUDA error code of its own.
int cuda_fail_msg(const char* where);

// Device-side error bits (OR-ed into the workspace status word).
enum : int { kErrSingular = 1, kErrNonfinite = 2, kErrTimeout = 4, kErrBounds = 8,
             kErrStructure = 16 /* a plan's coefficients no longer have its 2x2 structure */ };

// Forms of the equation (the block kernels' form parameter): Eq. (2.2), the
// d-term generalized form, and the paper's two-term form Eq. (3.1).
enum : int { kFormLaplace = 0, kFormDTerm = 1, kFormTwoTerm = 2 };

// Arithmetic used for the block products of a wavefront.
enum ProductKind : int { kProdNative = 0, kProdTF32 = 1, kProdBF16 = 2, kProdDMMA = 3 };

// Parameter block of one wavefront launch (passed by value).
struct WaveArgs {
    int nb[kMaxD];              // blocks per mode
    int hi[kMaxD];              // block updates read sources J' < hi[mu]
    long long tstride[kMaxD];   // linear block-grid stride of each mode
    const int* bsize[kMaxD];    // extent of every block (<= tile extent)
    const int* tiles;           // blocks of this wavefront (linear indices)
    int ntiles;
    int csize;                  // CTAs per block (cluster size)
    void* X;                    // block tensor: right-hand side in, solution out
    void* P[kMaxD];             // generalized form: P_l = X x_{eta>=l} C_eta  (l = 1..d-1)
    void* G[kMaxD];             //                   G_l = sum_{nu>=l} X x_nu A_nu x_{eta>=l,!=nu} C_eta
    const void* At[kMaxD];      // upper block triangle of A_mu, TE x TE tiles
    const void* Ct[kMaxD];      // same for C_mu (generalized form)
    int* err;                   // status word
    long long timeout_ns;       // bound of every device-side wait
    // persistent launches: per-block "solved" flags (nullptr: every source
    // block is already solved, as in a wavefront launch) and the launch-wide
    // abort word raised by a timed-out wait
    const int* ready;
    int* abort;
};

// Launch one wavefront.  T = double or float; generalized selects the d-term form.
template <typename T>
cudaError_t launch_wave(int d, bool generalized, int prod, const WaveArgs& a, cudaStream_t s);
// Raise the dynamic shared-memory limit of every wavefront kernel (call
// outside stream capture, once per process and device).
template <typename T>
cudaError_t prepare_wave();

// Workspace tables of one block partition (device pointers).
struct PartDev {
    const int* start[kMaxD];    // first index of every block
    const int* size[kMaxD];     // extent of every block
    const int* blk_of[kMaxD];   // block of every index
};

struct GeomArgs {
    int d;
    long long n[kMaxD];
    int nb[kMaxD];
    long long tstride[kMaxD];
    long long ntiles;
    PartDev part;
    int flip;                   // reverse every index (transposed solves)
};

// Layout conversions between the caller's column-major tensors and the block
// tensor (all dense tiles of TE^d entries, zero padded).
template <typename T>
cudaError_t launch_pack_tensor(const GeomArgs& g, const double* src, T* tiles, double scale, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack_tensor(const GeomArgs& g, const T* tiles, double* dst, cudaStream_t s);
// Coefficient tiles of mode mu: the upper block triangle (I <= J), tile (I, J)
// at index J (J + 1) / 2 + I.  upper_only: C (drop the subdiagonal).
template <typename T>
cudaError_t launch_pack_coef(const GeomArgs& g, int mu, const double* M, T* tiles, bool upper_only,
                             cudaStream_t s);
// Complex (interleaved) tensors and triangular coefficients.
cudaError_t launch_pack_tensor_z(const GeomArgs& g, const zd* src, zd* tiles, cudaStream_t s);
cudaError_t launch_unpack_tensor_z(const GeomArgs& g, const zd* tiles, zd* dst, cudaStream_t s);
cudaError_t launch_pack_coef_z(const GeomArgs& g, int mu, const zd* M, zd* tiles, cudaStream_t s);
// out[i] = sub-diagonal entries of every A_mu (concatenated, n_mu - 1 each).
cudaError_t launch_gather_subdiag(int d, const long long* n, const double* const* A, double* out,
                                  cudaStream_t s);
// Sets kErrStructure in *err unless the nonzero pattern of the first
// subdiagonal of every A_mu (modes back to back, entry i of mode mu: A(i+1, i))
// equals pat (one byte per entry).
cudaError_t launch_check_subdiag(int d, const long long* n, const double* const* A, const uint8_t* pat, int* err,
                                 cudaStream_t s);
// *status = the TSYLV status code of the device error word *err.
cudaError_t launch_status_word(const int* err, int* status, cudaStream_t s);

}  // namespace tsylv
