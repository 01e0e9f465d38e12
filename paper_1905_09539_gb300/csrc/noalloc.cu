// tsylv_solve_noalloc: the FP64 Laplace-form solve of tsylv_solve with every
// scratch buffer (status word, sub-diagonal read-back, schedule tables, block
// tensor, coefficient tiles) placed in one file-scope device array instead of
// a caller-provided workspace.
//
// It exists for callers that cannot allocate device memory when they solve:
// a host application whose own allocator owns all device memory, a real-time
// loop where cudaMalloc's latency and implicit synchronisation are not
// acceptable, or a plug-in that may not grow the process's device footprint
// after start-up.  Such a caller still passes its own inputs (A, B) and output
// (X); nothing else is needed.
//
// The array is fixed at kStaticScratchBytes; every GPU on which the library
// is loaded holds it until the process exits.  All calls share it and it keeps
// the previous call's contents, so calls whose GPU work overlaps (two host
// threads, or two streams without ordering between them) race on it and must
// be serialised by the caller.  The status word is cleared at the start of
// every call; everything else is fully written before it is read.
#include <cstring>
#include <mutex>
#include <vector>

#include "plan.h"
#include "solver.h"

namespace tsylv {

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_noalloc_mutex;
void* g_scratch_ptr[64] = {};

// Device address of the static scratch for the current device.  The first
// call on a device looks the address up (cudaGetSymbolAddress, with that
// device current) and raises the shared-memory limit of the kernels; later
// calls reuse both.  This set-up makes the first call on each device the one
// that should come before any stream capture.
int noalloc_scratch(char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return cuda_fail_msg("device index out of range for the static scratch table");
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        e = prepare_wave<double>();
        if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<char*>(g_scratch_ptr[dev]);
    return 0;
}

}  // namespace

int solver_solve_noalloc(int d, const int64_t* n, const double* const* A, const double* B, double* X,
                         const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    if (d < 1 || d > kMaxD) return -1;
    if (!solve_shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    if (!B) return -4;
    if (!X) return -5;
    // the option checks of tsylv_solve; then what this entry point serves:
    // the FP64 solve, without event timing
    if (int st = check_opts(o, d)) return st < 0 ? -6 : st;
    if (o.precision != TSYLV_FP64) return -6;
    // no event timing, no autotuning runs; FMA block updates
    if (o.timing || o.nmin < 0 || o.fp64_update == 2) return TSYLV_EUNSUPPORTED;
    // the largest workspace any admissible block structure needs must fit
    const size_t need = solver_workspace_bytes(d, n, false, o, false);
    if (need == 0) return -2;
    if (need > kStaticScratchBytes) {
        cuda_fail_msg("problem needs more scratch than the static array of tsylv_solve_noalloc (32 MiB)");
        return TSYLV_ESCRATCH;
    }
    char* base = nullptr;
    if (int st = noalloc_scratch(&base)) return st;
    (void)cudaGetLastError();

    long long nn[kMaxD];
    for (int mu = 0; mu < d; mu++) nn[mu] = n[mu];
    // 2x2 block structure of A (read back through the scratch), then the
    // schedule exactly as tsylv_solve plans it: block partition, wavefronts
    // (cluster split of short ones), device tables
    std::vector<uint8_t> sub;
    if (int st = solve_read_structure(d, nn, A, base, false, stream, sub)) return st;
    Plan p;
    fill_plan(p, d, nn, false, 8, o.split, sub, o.partition, shape_of_opts(o, d));
    cudaError_t e;
    Layout L = make_layout(d, nn, p.nb, false, 8, p.tab.size());
    if (L.total > kStaticScratchBytes) {
        cuda_fail_msg("problem needs more scratch than the static array of tsylv_solve_noalloc (32 MiB)");
        return TSYLV_ESCRATCH;
    }

    // queue the solve: status word, tables, coefficient tiles, block tensor,
    // wavefronts, solution
    GeomArgs g = geom_of(p, L, base, false);
    if ((e = cudaMemsetAsync(base + L.err, 0, 64, stream)) != cudaSuccess) return cuda_fail(e, "clear status");
    if ((e = cudaMemcpyAsync(base + L.tab, p.tab.data(), p.tab.size() * sizeof(int), cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess)
        return cuda_fail(e, "upload tables");
    for (int mu = 0; mu < d; mu++)
        if ((e = launch_pack_coef<double>(g, mu, A[mu], reinterpret_cast<double*>(base + L.At[mu]), false, stream)) !=
            cudaSuccess)
            return cuda_fail(e, "pack coefficients");
    double* Xt = reinterpret_cast<double*>(base + L.X);
    if ((e = launch_pack_tensor<double>(g, B, Xt, 1.0, stream)) != cudaSuccess) return cuda_fail(e, "pack B");
    WaveArgs wa{};
    const int* tab = reinterpret_cast<const int*>(base + L.tab);
    for (int mu = 0; mu < d; mu++) {
        wa.nb[mu] = p.nb[mu];
        wa.hi[mu] = p.nb[mu];
        wa.tstride[mu] = p.tstride[mu];
        wa.bsize[mu] = tab + p.t_size[mu];
        wa.At[mu] = base + L.At[mu];
    }
    wa.X = Xt;
    wa.err = reinterpret_cast<int*>(base + L.err);
    wa.timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (size_t w = 0; w < p.wave_off.size(); w++) {
        wa.tiles = tab + p.t_wave + p.wave_off[w];
        wa.ntiles = p.wave_cnt[w];
        wa.csize = p.wave_csize[w];
        if ((e = launch_wave<double>(d, false, kProdNative, wa, stream)) != cudaSuccess)
            return cuda_fail(e, "wavefront launch");
    }
    if ((e = launch_unpack_tensor<double>(g, Xt, X, stream)) != cudaSuccess) return cuda_fail(e, "unpack X");
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, base + L.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after solve");
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->waves = static_cast<int>(p.wave_off.size());
        info->launches = info->waves + d + 3;
        info->tiles = static_cast<int>(p.ntiles);
        for (int mu = 0; mu < d; mu++) info->leaf[mu] = shape_cut(d, mu, p.shape);
        info->resid = -1;
        info->norm_A = -1;
    }
    if (herr & kErrBounds) return cuda_fail_msg("device self-check: index outside a block array");
    if (herr & kErrTimeout) return TSYLV_ETIMEOUT;
    if (herr & kErrSingular) return TSYLV_ESINGULAR;
    if (herr & kErrNonfinite) return TSYLV_ENONFINITE;
    return TSYLV_OK;
}

}  // namespace tsylv

extern "C" int tsylv_solve_noalloc(int d, const int64_t* n, const double* const* A, const double* B, double* X,
                                   const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    return tsylv::solver_solve_noalloc(d, n, A, B, X, opts, info, stream);
}
