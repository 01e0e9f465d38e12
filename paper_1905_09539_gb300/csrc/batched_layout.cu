// Layout kernels of the batched solve (one launch for all equations) and the
// dispatch of the persistent kernel over (element type, d, form).
#include <type_traits>

#include "batched.h"

namespace tsylv {

template <typename T, int D, int GEN, int PK = kProdNative>
cudaError_t launch_batched_t(const BatchArgs& a, int grid, cudaStream_t s);
template <typename T, int D, int GEN, int PK = kProdNative>
cudaError_t prepare_batched_t();
template <typename T, int D, int GEN, int PK = kProdNative>
int batched_occupancy_t();

namespace {

// Column-major offset, in its equation's tensor, of in-block element e of a
// block with extents sz and first indices st (mode sizes n), the order D
// fixed at compile time (the tile extent a constant: no integer division);
// false for padding.
template <int D>
__device__ __forceinline__ bool tile_elem(int e, const int (&sz)[kMaxD], const long long (&st)[kMaxD],
                                          const long long* n, long long& off) {
    constexpr int TE = tile_extent(D);
    off = 0;
    long long gst = 1;
    bool valid = true;
#pragma unroll
    for (int mu = 0; mu < D; mu++) {
        const int i = e % TE;
        e /= TE;
        valid &= i < sz[mu];
        off += (st[mu] + i) * gst;
        gst *= n[mu];
    }
    return valid;
}

template <typename T, int D>
__device__ __forceinline__ void pack_tile(T* __restrict__ dst, const double* __restrict__ B, const BatchGeom& g,
                                          const int (&sz)[kMaxD], const long long (&st)[kMaxD]) {
    constexpr int TD = ipow(tile_extent(D), D);
    for (int e = threadIdx.x; e < TD; e += blockDim.x) {
        long long off;
        const bool v = tile_elem<D>(e, sz, st, g.n, off);
        dst[e] = v ? static_cast<T>(B[g.xoff + off]) : T(0);
    }
}

template <typename T, int D>
__device__ __forceinline__ void unpack_tile(const T* __restrict__ src, double* __restrict__ X, const BatchGeom& g,
                                            const int (&sz)[kMaxD], const long long (&st)[kMaxD]) {
    constexpr int TD = ipow(tile_extent(D), D);
    for (int e = threadIdx.x; e < TD; e += blockDim.x) {
        long long off;
        if (tile_elem<D>(e, sz, st, g.n, off)) X[g.xoff + off] = static_cast<double>(src[e]);
    }
}

// CTA b < njobs: block tensor tile of job b (B -> tile, zero padding);
// CTA njobs + c: coefficient tile c (A, and C for the generalized form;
// entries that the structure makes zero are written as zero unread).
template <typename T>
__global__ void k_batch_pack(const BatchGeom* __restrict__ geo, const BatchJob* __restrict__ jobs, int njobs,
                             const BatchCoefJob* __restrict__ cjobs, int ncjobs, const double* __restrict__ B,
                             const double* __restrict__ A, const double* __restrict__ C) {
    for (int b = blockIdx.x; b < njobs + ncjobs; b += gridDim.x) {
        if (b < njobs) {
            const BatchJob jb = jobs[b];
            const BatchGeom& g = geo[jb.eq];
            const int d = g.d, te = tile_extent(d), td = ipow(te, d);
            int sz[kMaxD] = {};
            long long st[kMaxD] = {};
            for (int mu = 0; mu < d; mu++) {
                const int I = static_cast<int>((jb.tile / g.tstride[mu]) % g.nb[mu]);
                sz[mu] = g.size[mu][I];
                st[mu] = g.start[mu][I];
            }
            T* dst = static_cast<T*>(g.X) + static_cast<long long>(jb.tile) * td;
            switch (d) {
                case 1: pack_tile<T, 1>(dst, B, g, sz, st); break;
                case 2: pack_tile<T, 2>(dst, B, g, sz, st); break;
                case 3: pack_tile<T, 3>(dst, B, g, sz, st); break;
                case 4: pack_tile<T, 4>(dst, B, g, sz, st); break;
                default: pack_tile<T, kMaxD>(dst, B, g, sz, st); break;
            }
        } else {
            const BatchCoefJob cj = cjobs[b - njobs];
            const BatchGeom& g = geo[cj.eq];
            const int te = tile_extent(g.d), tc = te * te, mu = cj.mu;
            const long long n = g.n[mu];
            const int si = g.size[mu][cj.I], sj = g.size[mu][cj.J];
            const long long gi0 = g.start[mu][cj.I], gj0 = g.start[mu][cj.J];
            const long long tri = static_cast<long long>(cj.J) * (cj.J + 1) / 2 + cj.I;
            T* ta = static_cast<T*>(g.At[mu]) + tri * tc;
            T* tcp = (C && g.Ct[mu]) ? static_cast<T*>(g.Ct[mu]) + tri * tc : nullptr;
            const double* Am = A + g.aoff[mu];
            const double* Cm = C ? C + g.aoff[mu] : nullptr;
            for (int e = threadIdx.x; e < tc; e += blockDim.x) {
                const int i = e % te, j = e / te;
                T va = T(0), vc = T(0);
                if (i < si && j < sj) {
                    const long long gi = gi0 + i, gj = gj0 + j;
                    if (gi <= gj + 1) va = static_cast<T>(Am[gi + n * gj]);
                    if (tcp && gi <= gj) vc = static_cast<T>(Cm[gi + n * gj]);
                }
                ta[e] = va;
                if (tcp) tcp[e] = vc;
            }
        }
    }
}

template <typename T>
__global__ void k_batch_unpack(const BatchGeom* __restrict__ geo, const BatchJob* __restrict__ jobs, int njobs,
                               double* __restrict__ X) {
    for (int b = blockIdx.x; b < njobs; b += gridDim.x) {
        const BatchJob jb = jobs[b];
        const BatchGeom& g = geo[jb.eq];
        const int d = g.d, te = tile_extent(d), td = ipow(te, d);
        int sz[kMaxD] = {};
        long long st[kMaxD] = {};
        for (int mu = 0; mu < d; mu++) {
            const int I = static_cast<int>((jb.tile / g.tstride[mu]) % g.nb[mu]);
            sz[mu] = g.size[mu][I];
            st[mu] = g.start[mu][I];
        }
        const T* src = static_cast<const T*>(g.X) + static_cast<long long>(jb.tile) * td;
        switch (d) {
            case 1: unpack_tile<T, 1>(src, X, g, sz, st); break;
            case 2: unpack_tile<T, 2>(src, X, g, sz, st); break;
            case 3: unpack_tile<T, 3>(src, X, g, sz, st); break;
            case 4: unpack_tile<T, 4>(src, X, g, sz, st); break;
            default: unpack_tile<T, kMaxD>(src, X, g, sz, st); break;
        }
    }
}

__global__ void k_batch_subdiag(const long long* __restrict__ aoff, const long long* __restrict__ nmat,
                                const long long* __restrict__ ooff, int nmats, const double* __restrict__ A,
                                double* __restrict__ out) {
    for (int k = blockIdx.y; k < nmats; k += gridDim.y) {
        const long long m = nmat[k];
        for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i + 1 < m;
             i += static_cast<long long>(gridDim.x) * blockDim.x)
            out[ooff[k] + i] = A[aoff[k] + (i + 1) + m * i];
    }
}

__global__ void k_store_args(const WaveArgs a, WaveArgs* dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = a;
}

inline int blocks_for(long long n) {
    long long b = n < 1 ? 1 : n;
    if (b > 152LL * 16) b = 152LL * 16;
    return static_cast<int>(b);
}

}  // namespace

template <typename T>
cudaError_t launch_batch_pack(const BatchGeom* g, const BatchJob* jobs, int njobs, const BatchCoefJob* cjobs,
                              int ncjobs, const double* B, const double* A, const double* C, cudaStream_t s) {
    k_batch_pack<T><<<blocks_for(static_cast<long long>(njobs) + ncjobs), 128, 0, s>>>(g, jobs, njobs, cjobs, ncjobs,
                                                                                      B, A, C);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_unpack(const BatchGeom* g, const BatchJob* jobs, int njobs, double* X, cudaStream_t s) {
    k_batch_unpack<T><<<blocks_for(njobs), 128, 0, s>>>(g, jobs, njobs, X);
    return cudaGetLastError();
}

cudaError_t launch_batch_subdiag(const long long* aoff, const long long* nmat, const long long* ooff, int nmats,
                                 long long maxn, const double* A, double* out, cudaStream_t s) {
    const unsigned gx = static_cast<unsigned>((maxn + 127) / 128 > 0 ? (maxn + 127) / 128 : 1);
    const unsigned gy = static_cast<unsigned>(nmats < 65535 ? (nmats > 0 ? nmats : 1) : 65535);
    k_batch_subdiag<<<dim3(gx, gy), 128, 0, s>>>(aoff, nmat, ooff, nmats, A, out);
    return cudaGetLastError();
}

cudaError_t launch_store_args(const WaveArgs& a, WaveArgs* dst, cudaStream_t s) {
    k_store_args<<<1, 32, 0, s>>>(a, dst);
    return cudaGetLastError();
}

namespace {

template <typename T, int PK>
cudaError_t launch_batched_pk(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return launch_batched_t<T, 1, false, PK>(a, grid, s);
        case 4: return launch_batched_t<T, 2, false, PK>(a, grid, s);
        case 5: return launch_batched_t<T, 2, true, PK>(a, grid, s);
        case 6: return launch_batched_t<T, 3, false, PK>(a, grid, s);
        case 7: return launch_batched_t<T, 3, true, PK>(a, grid, s);
        case 8: return launch_batched_t<T, 4, false, PK>(a, grid, s);
        case 9: return launch_batched_t<T, 4, true, PK>(a, grid, s);
        case 10: return launch_batched_t<T, 5, false, PK>(a, grid, s);  // d = 5: the Laplace form only
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int PK>
int batched_occupancy_pk(int d, bool gen) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return batched_occupancy_t<T, 1, false, PK>();
        case 4: return batched_occupancy_t<T, 2, false, PK>();
        case 5: return batched_occupancy_t<T, 2, true, PK>();
        case 6: return batched_occupancy_t<T, 3, false, PK>();
        case 7: return batched_occupancy_t<T, 3, true, PK>();
        case 8: return batched_occupancy_t<T, 4, false, PK>();
        case 9: return batched_occupancy_t<T, 4, true, PK>();
        case 10: return batched_occupancy_t<T, 5, false, PK>();
        default: return 1;
    }
}

template <typename T, int PK>
cudaError_t prepare_batched_pk() {
    cudaError_t e = cudaSuccess;
    if ((e = prepare_batched_t<T, 1, false, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 2, false, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 2, true, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 3, false, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 3, true, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 4, false, PK>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<T, 4, true, PK>()) != cudaSuccess) return e;
    return prepare_batched_t<T, 5, false, PK>();
}

// FP64 DMMA block updates: d = 2, 3 (tile extents 16 and 8 fill the 8 x 8
// output tiles; the 4-wide tiles of d >= 4 would leave half of each idle)
cudaError_t launch_batched_dmma(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 4: return launch_batched_t<double, 2, false, kProdDMMA>(a, grid, s);
        case 5: return launch_batched_t<double, 2, true, kProdDMMA>(a, grid, s);
        case 6: return launch_batched_t<double, 3, false, kProdDMMA>(a, grid, s);
        case 7: return launch_batched_t<double, 3, true, kProdDMMA>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batched_occupancy_dmma(int d, bool gen) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 4: return batched_occupancy_t<double, 2, false, kProdDMMA>();
        case 5: return batched_occupancy_t<double, 2, true, kProdDMMA>();
        case 6: return batched_occupancy_t<double, 3, false, kProdDMMA>();
        case 7: return batched_occupancy_t<double, 3, true, kProdDMMA>();
        default: return 1;
    }
}

cudaError_t prepare_batched_dmma() {
    cudaError_t e;
    if ((e = prepare_batched_t<double, 2, false, kProdDMMA>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<double, 2, true, kProdDMMA>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<double, 3, false, kProdDMMA>()) != cudaSuccess) return e;
    return prepare_batched_t<double, 3, true, kProdDMMA>();
}

}  // namespace

cudaError_t launch_batched_z(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return launch_batched_t<zd, 1, kFormLaplace>(a, grid, s);
        case 4: return launch_batched_t<zd, 2, kFormLaplace>(a, grid, s);
        case 5: return launch_batched_t<zd, 2, kFormDTerm>(a, grid, s);
        case 6: return launch_batched_t<zd, 3, kFormLaplace>(a, grid, s);
        case 7: return launch_batched_t<zd, 3, kFormDTerm>(a, grid, s);
        case 8: return launch_batched_t<zd, 4, kFormLaplace>(a, grid, s);
        case 9: return launch_batched_t<zd, 4, kFormDTerm>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batched_occupancy_z(int d, bool gen) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return batched_occupancy_t<zd, 1, kFormLaplace>();
        case 4: return batched_occupancy_t<zd, 2, kFormLaplace>();
        case 5: return batched_occupancy_t<zd, 2, kFormDTerm>();
        case 6: return batched_occupancy_t<zd, 3, kFormLaplace>();
        case 7: return batched_occupancy_t<zd, 3, kFormDTerm>();
        case 8: return batched_occupancy_t<zd, 4, kFormLaplace>();
        case 9: return batched_occupancy_t<zd, 4, kFormDTerm>();
        default: return 1;
    }
}

cudaError_t prepare_batched_z() {
    cudaError_t e;
    if ((e = prepare_batched_t<zd, 1, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<zd, 2, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<zd, 2, kFormDTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<zd, 3, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<zd, 3, kFormDTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<zd, 4, kFormLaplace>()) != cudaSuccess) return e;
    return prepare_batched_t<zd, 4, kFormDTerm>();
}

// The double-float solve (TSYLV_DF64): d = 1..4, Laplace and d-term forms.
cudaError_t launch_batched_df(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return launch_batched_t<dfl, 1, kFormLaplace>(a, grid, s);
        case 4: return launch_batched_t<dfl, 2, kFormLaplace>(a, grid, s);
        case 5: return launch_batched_t<dfl, 2, kFormDTerm>(a, grid, s);
        case 6: return launch_batched_t<dfl, 3, kFormLaplace>(a, grid, s);
        case 7: return launch_batched_t<dfl, 3, kFormDTerm>(a, grid, s);
        case 8: return launch_batched_t<dfl, 4, kFormLaplace>(a, grid, s);
        case 9: return launch_batched_t<dfl, 4, kFormDTerm>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batched_occupancy_df(int d, bool gen) {
    switch (d * 2 + (gen ? 1 : 0)) {
        case 2:
        case 3: return batched_occupancy_t<dfl, 1, kFormLaplace>();
        case 4: return batched_occupancy_t<dfl, 2, kFormLaplace>();
        case 5: return batched_occupancy_t<dfl, 2, kFormDTerm>();
        case 6: return batched_occupancy_t<dfl, 3, kFormLaplace>();
        case 7: return batched_occupancy_t<dfl, 3, kFormDTerm>();
        case 8: return batched_occupancy_t<dfl, 4, kFormLaplace>();
        case 9: return batched_occupancy_t<dfl, 4, kFormDTerm>();
        default: return 1;
    }
}

cudaError_t prepare_batched_df() {
    cudaError_t e;
    if ((e = prepare_batched_t<dfl, 1, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 2, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 2, kFormDTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 3, kFormLaplace>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 3, kFormDTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 4, kFormLaplace>()) != cudaSuccess) return e;
    return prepare_batched_t<dfl, 4, kFormDTerm>();
}

cudaError_t launch_batched_tt_df(int d, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d) {
        case 2: return launch_batched_t<dfl, 2, kFormTwoTerm>(a, grid, s);
        case 3: return launch_batched_t<dfl, 3, kFormTwoTerm>(a, grid, s);
        case 4: return launch_batched_t<dfl, 4, kFormTwoTerm>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batched_occupancy_tt_df(int d) {
    switch (d) {
        case 2: return batched_occupancy_t<dfl, 2, kFormTwoTerm>();
        case 3: return batched_occupancy_t<dfl, 3, kFormTwoTerm>();
        case 4: return batched_occupancy_t<dfl, 4, kFormTwoTerm>();
        default: return 1;
    }
}

cudaError_t prepare_batched_tt_df() {
    cudaError_t e;
    if ((e = prepare_batched_t<dfl, 2, kFormTwoTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<dfl, 3, kFormTwoTerm>()) != cudaSuccess) return e;
    return prepare_batched_t<dfl, 4, kFormTwoTerm>();
}

cudaError_t launch_batched_tt(int d, const BatchArgs& a, int grid, cudaStream_t s) {
    switch (d) {
        case 2: return launch_batched_t<double, 2, kFormTwoTerm>(a, grid, s);
        case 3: return launch_batched_t<double, 3, kFormTwoTerm>(a, grid, s);
        case 4: return launch_batched_t<double, 4, kFormTwoTerm>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int batched_occupancy_tt(int d) {
    switch (d) {
        case 2: return batched_occupancy_t<double, 2, kFormTwoTerm>();
        case 3: return batched_occupancy_t<double, 3, kFormTwoTerm>();
        case 4: return batched_occupancy_t<double, 4, kFormTwoTerm>();
        default: return 1;
    }
}

cudaError_t prepare_batched_tt() {
    cudaError_t e;
    if ((e = prepare_batched_t<double, 2, kFormTwoTerm>()) != cudaSuccess) return e;
    if ((e = prepare_batched_t<double, 3, kFormTwoTerm>()) != cudaSuccess) return e;
    return prepare_batched_t<double, 4, kFormTwoTerm>();
}

template <typename T>
cudaError_t launch_batched(int d, bool gen, const BatchArgs& a, int grid, cudaStream_t s, int prod) {
    if constexpr (std::is_same<T, float>::value) {
        if (prod == kProdTF32) return launch_batched_pk<float, kProdTF32>(d, gen, a, grid, s);
        if (prod == kProdBF16) return launch_batched_pk<float, kProdBF16>(d, gen, a, grid, s);
    } else {
        if (prod == kProdDMMA) return launch_batched_dmma(d, gen, a, grid, s);
    }
    if (prod != kProdNative) return cudaErrorInvalidValue;
    return launch_batched_pk<T, kProdNative>(d, gen, a, grid, s);
}

template <typename T>
int batched_occupancy(int d, bool gen, int prod) {
    if constexpr (std::is_same<T, float>::value) {
        if (prod == kProdTF32) return batched_occupancy_pk<float, kProdTF32>(d, gen);
        if (prod == kProdBF16) return batched_occupancy_pk<float, kProdBF16>(d, gen);
    } else {
        if (prod == kProdDMMA) return batched_occupancy_dmma(d, gen);
    }
    return batched_occupancy_pk<T, kProdNative>(d, gen);
}

template <typename T>
cudaError_t prepare_batched() {
    cudaError_t e = prepare_batched_pk<T, kProdNative>();
    if constexpr (std::is_same<T, float>::value) {
        if (e == cudaSuccess) e = prepare_batched_pk<float, kProdTF32>();
        if (e == cudaSuccess) e = prepare_batched_pk<float, kProdBF16>();
    } else {
        if (e == cudaSuccess) e = prepare_batched_dmma();
    }
    return e;
}

template cudaError_t launch_batched<double>(int, bool, const BatchArgs&, int, cudaStream_t, int);
template int batched_occupancy<double>(int, bool, int);
template cudaError_t prepare_batched<double>();
template cudaError_t launch_batched<float>(int, bool, const BatchArgs&, int, cudaStream_t, int);
template int batched_occupancy<float>(int, bool, int);
template cudaError_t prepare_batched<float>();
template cudaError_t launch_batch_pack<double>(const BatchGeom*, const BatchJob*, int, const BatchCoefJob*, int,
                                               const double*, const double*, const double*, cudaStream_t);
template cudaError_t launch_batch_unpack<double>(const BatchGeom*, const BatchJob*, int, double*, cudaStream_t);
template cudaError_t launch_batch_pack<float>(const BatchGeom*, const BatchJob*, int, const BatchCoefJob*, int,
                                              const double*, const double*, const double*, cudaStream_t);
template cudaError_t launch_batch_pack<dfl>(const BatchGeom*, const BatchJob*, int, const BatchCoefJob*, int,
                                            const double*, const double*, const double*, cudaStream_t);
template cudaError_t launch_batch_unpack<dfl>(const BatchGeom*, const BatchJob*, int, double*, cudaStream_t);

}  // namespace tsylv
