// Layout kernels: column-major tensors <-> block tensors (dense, zero-padded
// TE^d tiles in block-grid order), coefficient tiles, sub-diagonal gather.
#include "tsylv_internal.h"

namespace tsylv {
namespace {

// Block tensor element (tile t, local e) <-> global index.  flip reverses
// every mode (the index flip J of the transposed solve).
template <typename T, typename S = double>
__global__ void k_pack_tensor(const GeomArgs g, const S* __restrict__ src, T* __restrict__ tiles,
                              double scale) {
    const int d = g.d;
    const int te = tile_extent(d);
    const int td = ipow(te, d);
    const long long total = g.ntiles * td;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long t = idx / td;
        int e = static_cast<int>(idx % td);
        long long off = 0, gst = 1;
        bool valid = true;
        for (int mu = 0; mu < d; mu++) {
            const int I = static_cast<int>((t / g.tstride[mu]) % g.nb[mu]);
            const int i = e % te;
            e /= te;
            if (i >= g.part.size[mu][I]) { valid = false; break; }
            long long gi = g.part.start[mu][I] + i;
            if (g.flip) gi = g.n[mu] - 1 - gi;
            off += gi * gst;
            gst *= g.n[mu];
        }
        tiles[idx] = valid ? static_cast<T>(src[off] * scale) : T(0);
    }
}

template <typename T, typename S = double>
__global__ void k_unpack_tensor(const GeomArgs g, const T* __restrict__ tiles, S* __restrict__ dst) {
    const int d = g.d;
    const int te = tile_extent(d);
    const int td = ipow(te, d);
    long long total = 1;
    for (int mu = 0; mu < d; mu++) total *= g.n[mu];
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        long long rem = idx, t = 0;
        int e = 0, est = 1;
        for (int mu = 0; mu < d; mu++) {
            long long gi = rem % g.n[mu];
            rem /= g.n[mu];
            if (g.flip) gi = g.n[mu] - 1 - gi;
            const int I = g.part.blk_of[mu][gi];
            t += I * g.tstride[mu];
            e += static_cast<int>(gi - g.part.start[mu][I]) * est;
            est *= te;
        }
        dst[idx] = static_cast<S>(tiles[t * td + e]);
    }
}

// Tile (I, J), I <= J, of the upper block triangle; entries that the
// structure makes zero (below the first subdiagonal of A, below the diagonal
// of C) are written as zero without being read.  With flip, the tile holds
// J M^T J: entry (i, j) = M(n-1-j, n-1-i).
template <typename T, typename S = double>
__global__ void k_pack_coef(const GeomArgs g, int mu, const S* __restrict__ M, T* __restrict__ tiles,
                            int upper_only) {
    const int te = tile_extent(g.d);
    const int tc = te * te;
    const int nb = g.nb[mu];
    const long long n = g.n[mu];
    const long long total = static_cast<long long>(nb) * nb * tc;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int e = static_cast<int>(idx % tc);
        const long long pr = idx / tc;
        const int I = static_cast<int>(pr % nb), J = static_cast<int>(pr / nb);
        if (I > J) continue;
        const int i = e % te, j = e / te;
        T v = T(0);
        if (i < g.part.size[mu][I] && j < g.part.size[mu][J]) {
            const long long gi = g.part.start[mu][I] + i, gj = g.part.start[mu][J] + j;
            const bool keep = upper_only ? (gi <= gj) : (gi <= gj + 1);
            if (keep) {
                const long long ri = g.flip ? n - 1 - gj : gi;
                const long long rj = g.flip ? n - 1 - gi : gj;
                v = static_cast<T>(M[ri + n * rj]);
            }
        }
        const long long tri = static_cast<long long>(J) * (J + 1) / 2 + I;
        tiles[tri * tc + e] = v;
    }
}

struct SubdiagArgs {
    int d;
    long long n[kMaxD];
    const double* A[kMaxD];
};

__global__ void k_gather_subdiag(const SubdiagArgs a, double* out) {
    long long base = 0;
    for (int mu = 0; mu < a.d; mu++) {
        const long long m = a.n[mu];
        for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i + 1 < m;
             i += static_cast<long long>(gridDim.x) * blockDim.x)
            out[base + i] = a.A[mu][(i + 1) + m * i];
        base += m > 0 ? m - 1 : 0;
    }
}

__global__ void k_check_subdiag(const SubdiagArgs a, const uint8_t* __restrict__ pat, int* err) {
    long long base = 0;
    bool bad = false;
    for (int mu = 0; mu < a.d; mu++) {
        const long long m = a.n[mu];
        for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i + 1 < m;
             i += static_cast<long long>(gridDim.x) * blockDim.x)
            if ((a.A[mu][(i + 1) + m * i] != 0.0) != (pat[base + i] != 0)) bad = true;
        base += m > 0 ? m - 1 : 0;
    }
    if (bad) atomicOr(err, kErrStructure);
}

// the order of map_err on the host: device self-check, structure, timeout,
// singular, non-finite
__global__ void k_status_word(const int* __restrict__ err, int* __restrict__ status) {
    const int e = *err;
    *status = (e & kErrBounds)      ? TSYLV_ECUDA
              : (e & kErrStructure) ? -3
              : (e & kErrTimeout)   ? TSYLV_ETIMEOUT
              : (e & kErrSingular)  ? TSYLV_ESINGULAR
              : (e & kErrNonfinite) ? TSYLV_ENONFINITE
                                    : TSYLV_OK;
}

inline int grid_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

}  // namespace

template <typename T>
cudaError_t launch_pack_tensor(const GeomArgs& g, const double* src, T* tiles, double scale, cudaStream_t s) {
    const long long total = g.ntiles * ipow(tile_extent(g.d), g.d);
    k_pack_tensor<T><<<grid_for(total), 256, 0, s>>>(g, src, tiles, scale);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack_tensor(const GeomArgs& g, const T* tiles, double* dst, cudaStream_t s) {
    long long total = 1;
    for (int mu = 0; mu < g.d; mu++) total *= g.n[mu];
    k_unpack_tensor<T><<<grid_for(total), 256, 0, s>>>(g, tiles, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_coef(const GeomArgs& g, int mu, const double* M, T* tiles, bool upper_only, cudaStream_t s) {
    const int te = tile_extent(g.d);
    const long long total = static_cast<long long>(g.nb[mu]) * g.nb[mu] * te * te;
    k_pack_coef<T><<<grid_for(total), 256, 0, s>>>(g, mu, M, tiles, upper_only ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_gather_subdiag(int d, const long long* n, const double* const* A, double* out, cudaStream_t s) {
    SubdiagArgs a{};
    a.d = d;
    long long mx = 1;
    for (int mu = 0; mu < d; mu++) {
        a.n[mu] = n[mu];
        a.A[mu] = A[mu];
        if (n[mu] > mx) mx = n[mu];
    }
    k_gather_subdiag<<<grid_for(mx), 256, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t launch_check_subdiag(int d, const long long* n, const double* const* A, const uint8_t* pat, int* err,
                                 cudaStream_t s) {
    SubdiagArgs a{};
    a.d = d;
    long long mx = 1;
    for (int mu = 0; mu < d; mu++) {
        a.n[mu] = n[mu];
        a.A[mu] = A[mu];
        if (n[mu] > mx) mx = n[mu];
    }
    k_check_subdiag<<<grid_for(mx), 256, 0, s>>>(a, pat, err);
    return cudaGetLastError();
}

cudaError_t launch_status_word(const int* err, int* status, cudaStream_t s) {
    k_status_word<<<1, 1, 0, s>>>(err, status);
    return cudaGetLastError();
}

// Complex tensors and coefficients (interleaved re, im): the same index maps;
// complex triangular coefficients keep the upper triangle only.
cudaError_t launch_pack_tensor_z(const GeomArgs& g, const zd* src, zd* tiles, cudaStream_t s) {
    const long long total = g.ntiles * ipow(tile_extent(g.d), g.d);
    k_pack_tensor<zd, zd><<<grid_for(total), 256, 0, s>>>(g, src, tiles, 1.0);
    return cudaGetLastError();
}

cudaError_t launch_unpack_tensor_z(const GeomArgs& g, const zd* tiles, zd* dst, cudaStream_t s) {
    long long total = 1;
    for (int mu = 0; mu < g.d; mu++) total *= g.n[mu];
    k_unpack_tensor<zd, zd><<<grid_for(total), 256, 0, s>>>(g, tiles, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_coef_z(const GeomArgs& g, int mu, const zd* M, zd* tiles, cudaStream_t s) {
    const int te = tile_extent(g.d);
    const long long total = static_cast<long long>(g.nb[mu]) * g.nb[mu] * te * te;
    k_pack_coef<zd, zd><<<grid_for(total), 256, 0, s>>>(g, mu, M, tiles, 1);
    return cudaGetLastError();
}

template cudaError_t launch_pack_tensor<double>(const GeomArgs&, const double*, double*, double, cudaStream_t);
template cudaError_t launch_pack_tensor<float>(const GeomArgs&, const double*, float*, double, cudaStream_t);
template cudaError_t launch_unpack_tensor<double>(const GeomArgs&, const double*, double*, cudaStream_t);
template cudaError_t launch_unpack_tensor<float>(const GeomArgs&, const float*, double*, cudaStream_t);
template cudaError_t launch_pack_coef<double>(const GeomArgs&, int, const double*, double*, bool, cudaStream_t);
template cudaError_t launch_pack_coef<float>(const GeomArgs&, int, const double*, float*, bool, cudaStream_t);
template cudaError_t launch_pack_tensor<dfl>(const GeomArgs&, const double*, dfl*, double, cudaStream_t);
template cudaError_t launch_unpack_tensor<dfl>(const GeomArgs&, const dfl*, double*, cudaStream_t);
template cudaError_t launch_pack_coef<dfl>(const GeomArgs&, int, const double*, dfl*, bool, cudaStream_t);

}  // namespace tsylv
