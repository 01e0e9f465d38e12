// Solve orchestration: structure read-back, schedule, graph capture/replay,
// mixed-precision refinement and the residual entry point.
#include "solver.h"
#include "grad.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "batched.h"
#include "fused.h"
#include "plan.h"
#include "refine.h"

namespace tsylv {

namespace {

constexpr long long kTimeoutNs = 2000000000LL;  // bound of every device-side wait

// Second stream and fork/join events of one device: work that overlaps the
// main sequence of a solve (captured into the same graph as a parallel branch).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

SideStream* side_stream() {
    static std::mutex m;
    static SideStream st[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(m);
    SideStream& x = st[dev];
    if (!x.s) {
        if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
    }
    return &x;
}

}  // namespace

// Private non-blocking stream on which CUDA graphs are captured (capture on
// the caller's stream is not possible when it is the legacy default stream).
cudaStream_t capture_stream() {
    static std::mutex m;
    static cudaStream_t s[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(m);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!s[dev]) cudaStreamCreateWithFlags(&s[dev], cudaStreamNonBlocking);
    return s[dev];
}

namespace {

// Upper bound of the block-table size for any admissible structure.
size_t tab_ints_bound(int d, const long long* n, const int* nb) {
    size_t t = 0, nt = 1;
    for (int mu = 0; mu < d; mu++) {
        t += 2 * static_cast<size_t>(nb[mu]) + static_cast<size_t>(n[mu]);
        nt *= static_cast<size_t>(nb[mu]);
    }
    return t + nt + 4 * nt;  // + the job queue of the pipelined refinement steps
}

bool shape_ok(int d, const int64_t* n) {
    if (d < 1 || d > kMaxD || !n) return false;
    long long N = 1;
    for (int mu = 0; mu < d; mu++) {
        if (n[mu] < 1 || n[mu] > (1 << 20)) return false;
        N *= n[mu];
        if (N > (1LL << 34)) return false;
    }
    return true;
}

int map_err(int e) {
    if (e & kErrBounds) return cuda_fail_msg("device self-check: index outside a block array");
    if (e & kErrTimeout) return TSYLV_ETIMEOUT;
    if (e & kErrSingular) return TSYLV_ESINGULAR;
    if (e & kErrNonfinite) return TSYLV_ENONFINITE;
    return TSYLV_OK;
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace of a refined solve / residual: the FP32 solve's layout followed by
// the FP64 block tensors (B, X, R), FP64 coefficient tiles, their float-pair
// splits (DF64 residual), the generalized residual's two ping-pong sets of
// intermediates, and the reduction records.
struct RefLayout {
    Layout L32;
    size_t Bt = 0, Xt = 0, Rt = 0, Xh = 0, Xl = 0;
    size_t A64[kMaxD] = {}, C64[kMaxD] = {}, Ah[kMaxD] = {}, Al[kMaxD] = {}, Ch[kMaxD] = {}, Cl[kMaxD] = {};
    size_t set[2][4] = {};
    size_t part = 0, xpart = 0, xstat = 0, nrm = 0, nA = 0;
    size_t w2args = 0, flags2 = 0, nrm1 = 0;  // pipelined first two steps
    size_t total = 0;
};

RefLayout make_ref_layout(int d, const long long* n, const int* nb, bool gen, size_t tab_ints) {
    RefLayout R;
    R.L32 = make_layout(d, n, nb, gen, 4, tab_ints);
    const int te = tile_extent(d);
    const size_t td = static_cast<size_t>(ipow(te, d)), tc = static_cast<size_t>(te) * te;
    size_t nt = 1;
    for (int mu = 0; mu < d; mu++) nt *= static_cast<size_t>(nb[mu]);
    size_t o = R.L32.total;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = al256(o + bytes);
        return at;
    };
    R.Bt = take(nt * td * 8);
    R.Xt = take(nt * td * 8);
    R.Rt = take(nt * td * 8);
    R.Xh = take(nt * td * 4);
    R.Xl = take(nt * td * 4);
    for (int mu = 0; mu < d; mu++) {
        const size_t ntri = static_cast<size_t>(nb[mu]) * (nb[mu] + 1) / 2;
        R.A64[mu] = take(ntri * tc * 8);
        R.Ah[mu] = take(ntri * tc * 4);
        R.Al[mu] = take(ntri * tc * 4);
        if (gen) {
            R.C64[mu] = take(ntri * tc * 8);
            R.Ch[mu] = take(ntri * tc * 4);
            R.Cl[mu] = take(ntri * tc * 4);
        }
    }
    if (gen && d >= 2)
        for (int k = 0; k < 2; k++)
            for (int j = 0; j < 4; j++) R.set[k][j] = take(nt * td * 8);
    R.part = take(nt * 2 * 8);
    R.xpart = take(nt * 8);
    R.xstat = take(nt * 2 * 8);
    R.nrm = take(8 * 8);
    R.nA = take(2 * kMaxD * 8);
    R.w2args = take(sizeof(WaveArgs));
    R.flags2 = take(nt * 2 * sizeof(int));
    R.nrm1 = take(8 * 8);
    R.total = o;
    return R;
}

struct Call {
    int d = 0;
    bool gen = false, flip = false, df = true;
    long long n[kMaxD] = {};
    const double* A[kMaxD] = {};
    const double* C[kMaxD] = {};
    const double* B = nullptr;
    double* X = nullptr;
    const double* Xin = nullptr;  // tsylv_residual: the X to evaluate
    double* Rout = nullptr;       // tsylv_residual: output R
    const uint8_t* pat = nullptr;  // plan execution: the plan's subdiagonal pattern (device)
    int* status_out = nullptr;     // plan execution: device int for the status code
    char* base = nullptr;
    std::shared_ptr<Plan> plan;
    Layout L;
    RefLayout R;
    bool timing = false;
    bool persistent = true;   // opts->schedule == 0
    int flow_grid = 0;        // CTAs of the persistent launch
    bool update = false;      // refinement step: residual updated from the FP32 correction
    bool first = false;       // first refinement step (X = 0 before it: X after it is s D exactly)
    int prod = kProdNative;   // arithmetic of the FP32 solve's block updates (native / TF32 / BF16 tensor cores)
    bool tt = false;          // the paper's two-term form Eq. (3.1): C[0] is its C (mode 1)
    long long timeout_ns = kTimeoutNs;  // bound of every device-side wait (opts->wait_ms)
    bool pipe = false;        // first two refinement steps pipelined in one launch (Laplace form)
    int pipe_grid = 0;
};

inline cudaError_t mark(const Call& c, int i, cudaStream_t s) {
    // External: inside stream capture this becomes an event-record node of the graph
    return c.timing ? cudaEventRecordWithFlags(c.plan->ev[i], s, cudaEventRecordExternal) : cudaSuccess;
}

#define TRY(x)                            \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

WaveArgs wave_args(const Plan& p, const Layout& L, char* base, long long timeout_ns) {
    WaveArgs wa{};
    const int* tab = reinterpret_cast<const int*>(base + L.tab);
    for (int mu = 0; mu < p.d; mu++) {
        wa.nb[mu] = p.nb[mu];
        wa.hi[mu] = p.nb[mu];
        wa.tstride[mu] = p.tstride[mu];
        wa.bsize[mu] = tab + p.t_size[mu];
        wa.At[mu] = base + L.At[mu];
        wa.Ct[mu] = p.gen || (p.tt && mu == 0) ? base + L.Ct[mu] : nullptr;
        wa.P[mu] = (p.gen || p.tt) && mu >= 1 ? base + L.P[mu] : nullptr;
        wa.G[mu] = p.gen && mu >= 1 ? base + L.G[mu] : nullptr;
    }
    wa.X = base + L.X;
    wa.err = reinterpret_cast<int*>(base + L.err);
    wa.timeout_ns = timeout_ns;
    return wa;
}

// The block schedule of one solve: one persistent dataflow launch (every
// block taken from a queue in wavefront order; a block's update waits, per
// source block, until that block is solved), or one launch per wavefront.
template <typename T>
cudaError_t enqueue_waves(const Call& c, const Layout& L, cudaStream_t s) {
    const Plan& p = *c.plan;
    char* base = c.base;
    WaveArgs wa = wave_args(p, L, base, c.timeout_ns);
    const int* tab = reinterpret_cast<const int*>(base + L.tab);
    if (c.persistent) {
        int* ctl = reinterpret_cast<int*>(base + L.fctl);
        int* flags = reinterpret_cast<int*>(base + L.flags);
        TRY(cudaMemsetAsync(ctl, 0, 64, s));
        TRY(cudaMemsetAsync(flags, 0, static_cast<size_t>(p.ntiles) * sizeof(int), s));
        wa.ready = flags;
        wa.abort = ctl + 1;
        wa.csize = 1;
        WaveArgs* dargs = reinterpret_cast<WaveArgs*>(base + L.fargs);
        TRY(launch_store_args(wa, dargs, s));
        BatchArgs ba{};
        ba.eqs = dargs;
        ba.jobs = nullptr;
        ba.tiles = tab + p.t_wave;
        ba.njobs = static_cast<int>(p.ntiles);
        ba.head = ctl;
        ba.done = nullptr;
        ba.abort = ctl + 1;
        ba.timeout_ns = c.timeout_ns;
        if (p.tt) {
            if constexpr (std::is_same<T, dfl>::value) return launch_batched_tt_df(p.d, ba, c.flow_grid, s);
            else return launch_batched_tt(p.d, ba, c.flow_grid, s);
        }
        if constexpr (std::is_same<T, zd>::value)
            return launch_batched_z(p.d, p.gen, ba, c.flow_grid, s);
        else if constexpr (std::is_same<T, dfl>::value)
            return launch_batched_df(p.d, p.gen, ba, c.flow_grid, s);
        else
            return launch_batched<T>(p.d, p.gen, ba, c.flow_grid, s, c.prod);
    }
    if constexpr (std::is_same<T, zd>::value || std::is_same<T, dfl>::value) {
        return cudaErrorInvalidValue;  // the complex and double-float solves run the persistent schedule only
    } else {
        for (size_t w = 0; w < p.wave_off.size(); w++) {
            wa.tiles = tab + p.t_wave + p.wave_off[w];
            wa.ntiles = p.wave_cnt[w];
            wa.csize = p.wave_csize[w];
            TRY(launch_wave<T>(p.d, p.gen, kProdNative, wa, s));
        }
        return cudaSuccess;
    }
}

// ---------------------------------------------------------------- FP64 solve

// The FP64 solve (T = double) and the double-float solve (T = dfl: every
// coefficient and right-hand-side entry split into a pair of floats, the
// solution summed back into doubles): 8-byte entries, the same layout.
template <typename T>
cudaError_t enqueue_fp64_t(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const Layout& L = c.L;
    char* base = c.base;
    GeomArgs g = geom_of(p, L, base, c.flip);
    TRY(mark(c, 0, s));
    TRY(cudaMemsetAsync(base + L.err, 0, 64, s));
    TRY(cudaMemcpyAsync(base + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int mu = 0; mu < p.d; mu++) {
        TRY(launch_pack_coef<T>(g, mu, c.A[mu], reinterpret_cast<T*>(base + L.At[mu]), false, s));
        if (p.gen) TRY(launch_pack_coef<T>(g, mu, c.C[mu], reinterpret_cast<T*>(base + L.Ct[mu]), true, s));
    }
    T* Xt = reinterpret_cast<T*>(base + L.X);
    TRY(launch_pack_tensor<T>(g, c.B, Xt, 1.0, s));
    TRY(mark(c, 1, s));
    TRY(enqueue_waves<T>(c, L, s));
    TRY(mark(c, 2, s));
    TRY(launch_unpack_tensor<T>(g, Xt, c.X, s));
    return mark(c, 3, s);
}

cudaError_t enqueue_fp64(const Call& c, cudaStream_t s) { return enqueue_fp64_t<double>(c, s); }

// A plan execution: the FP64 solve, preceded by the check of the
// coefficients' 2x2 structure against the plan's and followed by the status
// code written to the caller's device int.
template <typename T>
cudaError_t enqueue_plan_t(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    char* base = c.base;
    int* err = reinterpret_cast<int*>(base + c.L.err);
    TRY(mark(c, 0, s));
    TRY(cudaMemsetAsync(err, 0, 64, s));
    TRY(launch_check_subdiag(p.d, c.n, c.A, c.pat, err, s));
    GeomArgs g = geom_of(p, c.L, base, c.flip);
    TRY(cudaMemcpyAsync(base + c.L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int mu = 0; mu < p.d; mu++) {
        TRY(launch_pack_coef<T>(g, mu, c.A[mu], reinterpret_cast<T*>(base + c.L.At[mu]), false, s));
        if (p.gen) TRY(launch_pack_coef<T>(g, mu, c.C[mu], reinterpret_cast<T*>(base + c.L.Ct[mu]), true, s));
    }
    T* Xt = reinterpret_cast<T*>(base + c.L.X);
    TRY(launch_pack_tensor<T>(g, c.B, Xt, 1.0, s));
    TRY(enqueue_waves<T>(c, c.L, s));
    TRY(launch_unpack_tensor<T>(g, Xt, c.X, s));
    if (c.status_out) TRY(launch_status_word(err, c.status_out, s));
    return cudaSuccess;
}

// The paper's two-term form Eq. (3.1), FP64: A_mu tiles of every mode (the
// A_1 term and the chain factors A_2 .. A_d), C tiles of mode 1, the
// persistent solve (the two-term form of the block kernel).
template <typename T>
cudaError_t enqueue_tt_t(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const Layout& L = c.L;
    char* base = c.base;
    GeomArgs g = geom_of(p, L, base, false);
    TRY(mark(c, 0, s));
    TRY(cudaMemsetAsync(base + L.err, 0, 64, s));
    TRY(cudaMemcpyAsync(base + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int mu = 0; mu < p.d; mu++)
        TRY(launch_pack_coef<T>(g, mu, c.A[mu], reinterpret_cast<T*>(base + L.At[mu]), false, s));
    TRY(launch_pack_coef<T>(g, 0, c.C[0], reinterpret_cast<T*>(base + L.Ct[0]), true, s));
    T* Xt = reinterpret_cast<T*>(base + L.X);
    TRY(launch_pack_tensor<T>(g, c.B, Xt, 1.0, s));
    TRY(mark(c, 1, s));
    TRY(enqueue_waves<T>(c, L, s));
    TRY(mark(c, 2, s));
    TRY(launch_unpack_tensor<T>(g, Xt, c.X, s));
    return mark(c, 3, s);
}

// Complex FP64 solve (complex-triangular coefficients): complex coefficient
// tiles (upper triangle), the complex block tensor of B, the persistent solve.
cudaError_t enqueue_z(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const Layout& L = c.L;
    char* base = c.base;
    GeomArgs g = geom_of(p, L, base, false);
    TRY(mark(c, 0, s));
    TRY(cudaMemsetAsync(base + L.err, 0, 64, s));
    TRY(cudaMemcpyAsync(base + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int mu = 0; mu < p.d; mu++) {
        TRY(launch_pack_coef_z(g, mu, reinterpret_cast<const zd*>(c.A[mu]), reinterpret_cast<zd*>(base + L.At[mu]), s));
        if (p.gen)
            TRY(launch_pack_coef_z(g, mu, reinterpret_cast<const zd*>(c.C[mu]), reinterpret_cast<zd*>(base + L.Ct[mu]),
                                   s));
    }
    zd* Xt = reinterpret_cast<zd*>(base + L.X);
    TRY(launch_pack_tensor_z(g, reinterpret_cast<const zd*>(c.B), Xt, s));
    TRY(mark(c, 1, s));
    TRY(enqueue_waves<zd>(c, L, s));
    TRY(mark(c, 2, s));
    TRY(launch_unpack_tensor_z(g, Xt, reinterpret_cast<zd*>(c.X), s));
    return mark(c, 3, s);
}

// ------------------------------------------------- residual R = B - A(X) (tiles)

// R = B - A(X) in FP64-accurate arithmetic (FP64 or DF64), or, with c.update,
// R -= s A(D) in FP32 for the FP32 correction D of the step (X += s D, s the
// scale max|R| of the step's right-hand side): the residual of the corrected
// X without re-evaluating A(X).  The update is accurate to about 2^-24 |A| |s D|,
// far below the residual once the correction is small.
cudaError_t enqueue_residual(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    char* b = c.base;
    ApplyArgs a{};
    const bool up = c.update;
    // first step from X = 0: X = s D with s a power of two, so A(X) = s A(D)
    // is evaluated in DF64 on the float correction D itself
    const bool fst = c.first && c.df && !up;
    for (int mu = 0; mu < p.d; mu++) {
        a.nb[mu] = p.nb[mu];
        a.tstride[mu] = p.tstride[mu];
        if (up) {
            a.A[mu] = b + R.L32.At[mu];
            a.C[mu] = p.gen ? b + R.L32.Ct[mu] : nullptr;
        } else if (c.df) {
            a.A[mu] = b + R.Ah[mu];
            a.Al[mu] = b + R.Al[mu];
            a.C[mu] = p.gen ? b + R.Ch[mu] : nullptr;
            a.Cl[mu] = p.gen ? b + R.Cl[mu] : nullptr;
        } else {
            a.A[mu] = b + R.A64[mu];
            a.C[mu] = p.gen ? b + R.C64[mu] : nullptr;
        }
    }
    a.ntiles = p.ntiles;
    a.B = reinterpret_cast<const double*>(b + (up ? R.Rt : R.Bt));
    a.R = reinterpret_cast<double*>(b + R.Rt);
    a.scale = up || fst ? reinterpret_cast<const double*>(b + R.nrm) : nullptr;
    a.part = reinterpret_cast<double*>(b + R.part);
    a.err = reinterpret_cast<int*>(b + R.L32.err);
    a.timeout_ns = c.timeout_ns;
    const void* xs = up || fst ? static_cast<const void*>(b + R.L32.X)
                               : c.df ? static_cast<const void*>(b + R.Xh) : static_cast<const void*>(b + R.Xt);
    const void* xsl = c.df && !up && !fst ? static_cast<const void*>(b + R.Xl) : nullptr;
    auto launch = [&](const ApplyArgs& aa) {
        if (fst && aa.s1l == nullptr) return launch_apply_dfh(p.d, aa, s);  // the levels reading D
        return up ? launch_apply_f32(p.d, aa, s) : c.df ? launch_apply<true>(p.d, aa, s) : launch_apply<false>(p.d, aa, s);
    };
    if (!p.gen) {
        a.kind = kApplyLaplace;
        a.s1 = xs;
        a.s1l = xsl;
        return launch(a);
    }
    // Horner levels d-1 .. 0, ping-pong between the two intermediate sets
    int cur = 0;
    auto setp = [&](int k, int j) -> void* { return b + R.set[k][j]; };
    a.kind = kApplyFirst;
    a.mode = p.d - 1;
    a.s1 = xs;
    a.s1l = xsl;
    a.o1 = setp(0, 0);
    a.o1l = setp(0, 1);
    a.o2 = setp(0, 2);
    a.o2l = setp(0, 3);
    TRY(launch(a));
    for (int l = p.d - 2; l >= 0; l--) {
        a.kind = l == 0 ? kApplyFinal : kApplyMiddle;
        a.mode = l;
        a.s1 = setp(cur, 0);
        a.s1l = setp(cur, 1);
        a.s2 = setp(cur, 2);
        a.s2l = setp(cur, 3);
        a.o1 = setp(1 - cur, 0);
        a.o1l = setp(1 - cur, 1);
        a.o2 = setp(1 - cur, 2);
        a.o2l = setp(1 - cur, 3);
        TRY(launch(a));
        cur = 1 - cur;
    }
    return cudaSuccess;
}

// coefficient tiles of the residual (FP64, and their float-pair split)
cudaError_t enqueue_coef64(const Call& c, const GeomArgs& g, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    char* b = c.base;
    const long long tc = static_cast<long long>(p.tc);
    for (int mu = 0; mu < p.d; mu++) {
        const long long ntri = static_cast<long long>(p.nb[mu]) * (p.nb[mu] + 1) / 2;
        TRY(launch_pack_coef<double>(g, mu, c.A[mu], reinterpret_cast<double*>(b + R.A64[mu]), false, s));
        if (c.df)
            TRY(launch_split(reinterpret_cast<double*>(b + R.A64[mu]), reinterpret_cast<float*>(b + R.Ah[mu]),
                             reinterpret_cast<float*>(b + R.Al[mu]), ntri * tc, s));
        if (p.gen) {
            TRY(launch_pack_coef<double>(g, mu, c.C[mu], reinterpret_cast<double*>(b + R.C64[mu]), true, s));
            if (c.df)
                TRY(launch_split(reinterpret_cast<double*>(b + R.C64[mu]), reinterpret_cast<float*>(b + R.Ch[mu]),
                                 reinterpret_cast<float*>(b + R.Cl[mu]), ntri * tc, s));
        }
    }
    return cudaSuccess;
}

cudaError_t enqueue_norms(const Call& c, cudaStream_t s) {
    NormArgs na{};
    int cnt = 0, nmax = 1;
    for (int mu = 0; mu < c.d; mu++) {
        na.M[cnt] = c.A[mu];
        na.n[cnt] = static_cast<int>(c.n[mu]);
        na.upper[cnt++] = 0;
        nmax = std::max(nmax, static_cast<int>(c.n[mu]));
    }
    if (c.gen)
        for (int mu = 0; mu < c.d; mu++) {
            na.M[cnt] = c.C[mu];
            na.n[cnt] = static_cast<int>(c.n[mu]);
            na.upper[cnt++] = 1;
        }
    return launch_norm2(na, cnt, nmax, reinterpret_cast<double*>(c.base + c.R.nA), s);
}

// ---------------------------------------------------------- refined solve

cudaError_t enqueue_ref_setup(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    const Layout& L = R.L32;
    char* b = c.base;
    GeomArgs g = geom_of(p, L, b, c.flip);
    const long long nel = p.ntiles * p.td;
    TRY(cudaMemsetAsync(b + L.err, 0, 64, s));
    TRY(cudaMemcpyAsync(b + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int mu = 0; mu < p.d; mu++) {
        TRY(launch_pack_coef<float>(g, mu, c.A[mu], reinterpret_cast<float*>(b + L.At[mu]), false, s));
        if (p.gen) TRY(launch_pack_coef<float>(g, mu, c.C[mu], reinterpret_cast<float*>(b + L.Ct[mu]), true, s));
    }
    TRY(enqueue_coef64(c, g, s));
    TRY(launch_pack_tensor<double>(g, c.B, reinterpret_cast<double*>(b + R.Bt), 1.0, s));
    TRY(cudaMemcpyAsync(b + R.Rt, b + R.Bt, nel * 8, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemsetAsync(b + R.Xt, 0, nel * 8, s));
    TRY(cudaMemsetAsync(b + R.Xh, 0, nel * 4, s));
    TRY(cudaMemsetAsync(b + R.Xl, 0, nel * 4, s));
    TRY(launch_tile_stats(reinterpret_cast<double*>(b + R.Rt), reinterpret_cast<double*>(b + R.part), p.ntiles, p.td,
                          s));
    return launch_reduce(reinterpret_cast<double*>(b + R.part), nullptr, p.ntiles,
                         reinterpret_cast<double*>(b + R.nrm), s);
}

cudaError_t enqueue_ref_iter(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    const Layout& L = R.L32;
    char* b = c.base;
    const long long nel = p.ntiles * p.td;
    const double* nrm = reinterpret_cast<const double*>(b + R.nrm);
    TRY(mark(c, 0, s));
    // a full step also estimates the coefficient norms (they scale the
    // stopping test), on a parallel branch that overlaps the FP32 solve
    SideStream* side = c.update ? nullptr : side_stream();
    if (!c.update) {
        if (side) {
            TRY(cudaEventRecord(side->fork, s));
            TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
            TRY(enqueue_norms(c, side->s));
            TRY(cudaEventRecord(side->join, side->s));
        } else {
            TRY(enqueue_norms(c, s));
        }
    }
    // low-precision solve of A(D) = R / max|R|
    TRY(launch_scale_to_f32(reinterpret_cast<double*>(b + R.Rt), reinterpret_cast<float*>(b + L.X), nrm, nel, s));
    TRY(enqueue_waves<float>(c, L, s));
    // X += max|R| D  (FP64), its float-pair split, block sums of X^2
    // the float-pair X only feeds a full DF64 residual of a later step
    const bool split = c.df && !c.update && !c.first;
    TRY(launch_update_x(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<float*>(b + L.X), nrm,
                        split ? reinterpret_cast<float*>(b + R.Xh) : nullptr,
                        split ? reinterpret_cast<float*>(b + R.Xl) : nullptr, reinterpret_cast<double*>(b + R.xpart),
                        nel, p.td, s));
    TRY(mark(c, 1, s));
    // R = B - A(X) in FP64-accurate arithmetic, or R -= s A(D) in FP32
    TRY(enqueue_residual(c, s));
    TRY(mark(c, 2, s));
    if (side) TRY(cudaStreamWaitEvent(s, side->join, 0));
    TRY(launch_reduce(reinterpret_cast<double*>(b + R.part), reinterpret_cast<double*>(b + R.xpart), p.ntiles,
                      reinterpret_cast<double*>(b + R.nrm), s));
    return mark(c, 3, s);
}

// First two refinement steps (Laplace form) in one pipelined launch: the
// second FP32 solve, and both residuals, follow the first solve block by
// block instead of waiting for it to finish (see Refine2Args).  The same
// arithmetic as two separate steps: R1 = B - s A(D1) in double-float on the
// float correction, D2 = solve(R1 / s), R2 = R1 - s A(D2) in FP32, X = s D1 + s D2
// (the second step's scale s is the first's: power-of-two scalings are exact).
cudaError_t enqueue_ref_pipe(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    const Layout& L = R.L32;
    char* b = c.base;
    const long long nel = p.ntiles * p.td;
    double* nrm = reinterpret_cast<double*>(b + R.nrm);
    TRY(mark(c, 0, s));
    SideStream* side = side_stream();
    if (side) {
        TRY(cudaEventRecord(side->fork, s));
        TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
        TRY(enqueue_norms(c, side->s));
        TRY(cudaEventRecord(side->join, side->s));
    } else {
        TRY(enqueue_norms(c, s));
    }
    TRY(launch_scale_to_f32(reinterpret_cast<double*>(b + R.Rt), reinterpret_cast<float*>(b + L.X), nrm, nel, s));
    int* ctl = reinterpret_cast<int*>(b + L.fctl);
    int* flags1 = reinterpret_cast<int*>(b + L.flags);
    int* flags2 = reinterpret_cast<int*>(b + R.flags2);  // [r1done | s2done]
    TRY(cudaMemsetAsync(ctl, 0, 64, s));
    TRY(cudaMemsetAsync(flags1, 0, static_cast<size_t>(p.ntiles) * sizeof(int), s));
    TRY(cudaMemsetAsync(flags2, 0, static_cast<size_t>(p.ntiles) * 2 * sizeof(int), s));
    WaveArgs w1 = wave_args(p, L, b, c.timeout_ns);
    w1.ready = flags1;
    w1.abort = ctl + 1;
    w1.csize = 1;
    WaveArgs w2 = w1;
    w2.X = b + R.Xh;  // the second solve's right-hand side / solution (the float split is not needed here)
    w2.ready = flags2 + p.ntiles;
    WaveArgs* d1 = reinterpret_cast<WaveArgs*>(b + L.fargs);
    WaveArgs* d2 = reinterpret_cast<WaveArgs*>(b + R.w2args);
    TRY(launch_store_args(w1, d1, s));
    TRY(launch_store_args(w2, d2, s));
    Refine2Args f{};
    f.w1 = d1;
    f.w2 = d2;
    f.jobs = reinterpret_cast<const int*>(b + L.tab) + p.t_rjobs;
    f.njobs = p.n_rjobs;
    f.head = ctl;
    f.abort = ctl + 1;
    f.timeout_ns = c.timeout_ns;
    f.r1done = flags2;
    for (ApplyArgs* ap : {&f.r1, &f.r2}) {
        for (int mu = 0; mu < p.d; mu++) {
            ap->nb[mu] = p.nb[mu];
            ap->tstride[mu] = p.tstride[mu];
        }
        ap->ntiles = p.ntiles;
        ap->kind = kApplyLaplace;
        ap->R = reinterpret_cast<double*>(b + R.Rt);
        ap->scale = nrm;
        ap->err = reinterpret_cast<int*>(b + L.err);
        ap->timeout_ns = c.timeout_ns;
    }
    for (int mu = 0; mu < p.d; mu++) {
        f.r1.A[mu] = b + R.Ah[mu];
        f.r1.Al[mu] = b + R.Al[mu];
        f.r2.A[mu] = b + L.At[mu];
    }
    f.r1.s1 = b + L.X;
    f.r1.B = reinterpret_cast<const double*>(b + R.Bt);
    f.r1.part = reinterpret_cast<double*>(b + R.xstat);  // the first residual's block norms
    f.r2.s1 = b + R.Xh;
    f.r2.B = reinterpret_cast<const double*>(b + R.Rt);  // updated in place
    f.r2.part = reinterpret_cast<double*>(b + R.part);
    f.X2 = reinterpret_cast<float*>(b + R.Xh);
    f.nrm = nrm;
    // timing marks: 0 -> 1 both solves with their residuals, 1 -> 2 the X update
    TRY(launch_refine2(p.d, c.prod, f, c.pipe_grid, s));
    TRY(mark(c, 1, s));
    // X = s D1 + s D2 (FP64), block sums of X^2
    double* xpart = reinterpret_cast<double*>(b + R.xpart);
    TRY(launch_update_x(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<float*>(b + L.X), nrm, nullptr, nullptr,
                        xpart, nel, p.td, s));
    TRY(launch_update_x(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<float*>(b + R.Xh), nrm, nullptr, nullptr,
                        xpart, nel, p.td, s));
    TRY(mark(c, 2, s));
    if (side) TRY(cudaStreamWaitEvent(s, side->join, 0));
    TRY(launch_reduce(reinterpret_cast<double*>(b + R.xstat), nullptr, p.ntiles, reinterpret_cast<double*>(b + R.nrm1),
                      s));
    TRY(launch_reduce(reinterpret_cast<double*>(b + R.part), xpart, p.ntiles, nrm, s));
    return mark(c, 3, s);
}

// The full FP64-accurate residual of the current X (after the pipelined steps,
// where separate steps would have re-evaluated the second residual in full).
cudaError_t enqueue_ref_resid_full(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    char* b = c.base;
    const long long nel = p.ntiles * p.td;
    if (c.df)
        TRY(launch_split(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<float*>(b + R.Xh),
                         reinterpret_cast<float*>(b + R.Xl), nel, s));
    TRY(enqueue_residual(c, s));
    return launch_reduce(reinterpret_cast<double*>(b + R.part), reinterpret_cast<double*>(b + R.xpart), p.ntiles,
                         reinterpret_cast<double*>(b + R.nrm), s);
}

cudaError_t enqueue_ref_final(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    GeomArgs g = geom_of(p, c.R.L32, c.base, c.flip);
    return launch_unpack_tensor<double>(g, reinterpret_cast<double*>(c.base + c.R.Xt), c.X, s);
}

// ------------------------------------------------------------- residual API

cudaError_t enqueue_resid_api(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const RefLayout& R = c.R;
    const Layout& L = R.L32;
    char* b = c.base;
    GeomArgs g = geom_of(p, L, b, false);
    const long long nel = p.ntiles * p.td;
    TRY(cudaMemsetAsync(b + L.err, 0, 64, s));
    TRY(cudaMemcpyAsync(b + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    TRY(enqueue_coef64(c, g, s));
    TRY(launch_pack_tensor<double>(g, c.B, reinterpret_cast<double*>(b + R.Bt), 1.0, s));
    TRY(launch_pack_tensor<double>(g, c.Xin, reinterpret_cast<double*>(b + R.Xt), 1.0, s));
    if (c.df)
        TRY(launch_split(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<float*>(b + R.Xh),
                         reinterpret_cast<float*>(b + R.Xl), nel, s));
    TRY(launch_tile_stats(reinterpret_cast<double*>(b + R.Xt), reinterpret_cast<double*>(b + R.xstat), p.ntiles, p.td,
                          s));
    TRY(launch_reduce(reinterpret_cast<double*>(b + R.xstat), nullptr, p.ntiles,
                      reinterpret_cast<double*>(b + R.nrm) + 4, s));
    TRY(enqueue_residual(c, s));
    TRY(launch_reduce(reinterpret_cast<double*>(b + R.part), nullptr, p.ntiles, reinterpret_cast<double*>(b + R.nrm),
                      s));
    TRY(enqueue_norms(c, s));
    return launch_unpack_tensor<double>(g, reinterpret_cast<double*>(b + R.Rt), c.Rout, s);
}

// ---------------------------------------------------------- graph runner

int run_enqueue(Plan& p, const std::vector<const void*>& key, bool use_graph, cudaStream_t stream,
                cudaError_t (*fn)(const Call&, cudaStream_t), const Call& c) {
    cudaError_t e;
    if (!use_graph) {
        if ((e = fn(c, stream)) != cudaSuccess) return cuda_fail(e, "enqueue");
        return 0;
    }
    static std::mutex gm;
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(gm);
        for (auto& ge : p.graphs)
            if (ge.key == key) exec = ge.exec;
        if (!exec) {
            cudaStream_t cs = capture_stream();
            if (!cs) return cuda_fail_msg("capture stream");
            if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamBeginCapture");
            e = fn(c, cs);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e != cudaSuccess ? e : e2, e != cudaSuccess ? "capture: enqueue" : "cudaStreamEndCapture");
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            if (p.graphs.size() >= 32) {
                cudaGraphExecDestroy(p.graphs.front().exec);
                p.graphs.erase(p.graphs.begin());
            }
            p.graphs.push_back(GraphEntry{key, exec});
        }
    }
    if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return 0;
}

// CTAs of a persistent launch: every resident slot of the GPU, at most one per block.
int flow_grid(int elem, int d, bool gen, long long ntiles, int prod = kProdNative) {
    static std::mutex m;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const int key = (((dev * 2 + (elem == 4 ? 1 : 0)) * 8 + d) * 2 + (gen ? 1 : 0)) * 4 + prod;
    int slots = 0;
    {
        std::lock_guard<std::mutex> lk(m);
        auto it = cache.find(key);
        if (it != cache.end()) {
            slots = it->second;
        } else {
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
            const int occ = elem == 4 ? batched_occupancy<float>(d, gen, prod) : batched_occupancy<double>(d, gen, prod);
            slots = sms * occ;
            cache[key] = slots;
        }
    }
    return static_cast<int>(ntiles < slots ? ntiles : slots);
}

// CTAs of the pipelined first two refinement steps.
int pipe_grid(int d, long long ntiles, int prod) {
    static std::mutex m;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const int key = (dev * 8 + d) * 4 + prod;
    int slots = 0;
    {
        std::lock_guard<std::mutex> lk(m);
        auto it = cache.find(key);
        if (it != cache.end()) {
            slots = it->second;
        } else {
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
            slots = sms * refine2_occupancy(d, prod);
            cache[key] = slots;
        }
    }
    return static_cast<int>(ntiles < slots ? ntiles : slots);
}

int prepare_kernels() {
    static std::mutex pm;
    static bool prepared[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(pm);
    if (dev >= 0 && dev < 64 && !prepared[dev]) {
        cudaError_t e = prepare_wave<double>();
        if (e == cudaSuccess) e = prepare_wave<float>();
        if (e == cudaSuccess) e = prepare_apply<false>();
        if (e == cudaSuccess) e = prepare_apply<true>();
        if (e == cudaSuccess) e = prepare_apply_f32();
        if (e == cudaSuccess) e = prepare_apply_dfh();
        if (e == cudaSuccess) e = prepare_batched<double>();
        if (e == cudaSuccess) e = prepare_batched<float>();
        if (e == cudaSuccess) e = prepare_batched_tt();
        if (e == cudaSuccess) e = prepare_batched_z();
        if (e == cudaSuccess) e = prepare_batched_df();
        if (e == cudaSuccess) e = prepare_batched_tt_df();
        if (e == cudaSuccess) e = prepare_refine2();
        if (e == cudaSuccess) e = prepare_norm2();
        if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
        prepared[dev] = true;
    }
    return 0;
}

// 2x2 block structure of every A_mu (sub-diagonal read back through the
// workspace), validated; flipped for the transposed equation.
int read_structure(int d, const long long* n, const double* const* A, char* base, bool flip, cudaStream_t stream,
                   std::vector<uint8_t>& sub) {
    size_t nsub = 0;
    for (int mu = 0; mu < d; mu++) nsub += static_cast<size_t>(n[mu] - 1);
    std::vector<double> hsub(nsub + 1, 0.0);
    const size_t sub_off = 256;  // Layout::sub does not depend on the block counts
    double* dsub = reinterpret_cast<double*>(base + sub_off);
    cudaError_t e;
    if (nsub > 0) {
        if ((e = launch_gather_subdiag(d, n, A, dsub, stream)) != cudaSuccess) return cuda_fail(e, "gather sub-diagonal");
        if ((e = cudaMemcpyAsync(hsub.data(), dsub, nsub * sizeof(double), cudaMemcpyDeviceToHost, stream)) !=
            cudaSuccess)
            return cuda_fail(e, "read sub-diagonal");
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize before planning");
    sub.assign(nsub + 1, 0);
    size_t off = 0;
    for (int mu = 0; mu < d; mu++) {
        const long long m = n[mu];
        for (long long i = 0; i + 1 < m; i++) {
            const size_t src = flip ? off + static_cast<size_t>(m - 2 - i) : off + static_cast<size_t>(i);
            sub[off + i] = hsub[src] != 0.0 ? 1 : 0;
        }
        for (long long i = 0; i + 2 < m; i++)
            if (sub[off + i] && sub[off + i + 1]) return -3;  // not quasi-triangular
        off += static_cast<size_t>(m - 1);
    }
    return 0;
}

std::vector<const void*> make_key(const Call& c, int tag) {
    std::vector<const void*> key;
    for (int mu = 0; mu < c.d; mu++) {
        key.push_back(c.A[mu]);
        key.push_back(c.C[mu]);
    }
    key.push_back(c.B);
    key.push_back(c.X);
    key.push_back(c.Xin);
    key.push_back(c.Rout);
    key.push_back(c.status_out);
    key.push_back(c.base);
    key.push_back(reinterpret_cast<const void*>(static_cast<uintptr_t>(tag)));
    key.push_back(reinterpret_cast<const void*>(static_cast<uintptr_t>(c.timeout_ns)));
    return key;
}

int ensure_events(Call& c) {
    if (c.timing && !c.plan->ev[0])
        for (auto& ev : c.plan->ev)
            if (cudaError_t e = cudaEventCreate(&ev); e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    return 0;
}

double norm_op(const Call& c, const double* nA) {
    double s = 0;
    for (int mu = 0; mu < c.d; mu++) {
        double t = nA[mu];
        if (c.gen)
            for (int eta = 0; eta < c.d; eta++)
                if (eta != mu) t *= nA[c.d + eta];
        s += t;
    }
    return s;
}

}  // namespace

bool solve_shape_ok(int d, const int64_t* n) { return shape_ok(d, n); }

int solve_read_structure(int d, const long long* n, const double* const* A, char* base, bool flip,
                         cudaStream_t stream, std::vector<uint8_t>& sub) {
    return read_structure(d, n, A, base, flip, stream, sub);
}

int check_opts(const tsylv_opts& o, int d) {
    if (o.precision < TSYLV_FP64 || o.precision > TSYLV_DF64 || o.max_refine < 0 || !(o.tol > 0) ||
        (o.residual != TSYLV_RESID_DF64 && o.residual != TSYLV_RESID_FP64) || o.split < 0 || o.nmin < -1 ||
        o.schedule < 0 || o.schedule > 1 || o.partition < 0 || o.partition > 1 || o.resid_update < 0 ||
        o.resid_update > 1 || o.fuse_step < 0 || o.fuse_step > 3 || o.timing < 0 || o.timing > 1 ||
        o.use_graph < 0 || o.use_graph > 1 || o.wait_ms < 1 || o.wait_ms > 600000 || o.fp64_update < 0 ||
        o.fp64_update > 2)
        return -1;
    if (o.nmin < -1) return -1;
    for (int mu = 0; mu < kMaxD; mu++)
        if (o.leaf[mu] < 0) return -1;
    if (o.host_io || o.nmin == 1 || o.nmin > tile_extent(d)) return TSYLV_EUNSUPPORTED;
    for (int mu = 0; mu < d; mu++)
        if (o.leaf[mu] == 1 || o.leaf[mu] > tile_extent(d)) return TSYLV_EUNSUPPORTED;
    // fuse_step 1 (the first step as one launch) is no longer offered: it
    // measured slower than separate launches
    if (o.fuse_step == 1) return TSYLV_EUNSUPPORTED;
    return 0;
}

// Block-update arithmetic of a TSYLV_FP64 solve (opts->fp64_update): FMA by
// default; DMMA on request, built for d = 2, 3 in the Laplace and d-term forms
// on the persistent schedule (-1: asked for where it is not built).
int fp64_prod(const tsylv_opts& o, int d, bool persistent) {
    if (o.fp64_update != 2) return kProdNative;
    return (d == 2 || d == 3) && persistent ? kProdDMMA : -1;
}

int shape_of_nmin(int nmin) { return nmin == 0 ? 0 : nmin > 0 ? kShapeFixed + nmin : -1; }

int shape_of_opts(const tsylv_opts& o, int d) {
    bool per_mode = false;
    for (int mu = 0; mu < d; mu++) per_mode |= o.leaf[mu] > 0;
    if (!per_mode) return shape_of_nmin(o.nmin);
    const int dflt = o.nmin > 0 ? o.nmin : tile_extent(d);
    int code = 0;
    for (int mu = 0; mu < d; mu++) code |= (o.leaf[mu] > 0 ? o.leaf[mu] : dflt) << (6 * mu);
    return kShapeFixed + code;
}

size_t solver_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o, bool transposed) {
    (void)transposed;
    if (!shape_ok(d, n)) return 0;
    long long nn[kMaxD];
    int nb[kMaxD];
    const int shape = shape_of_opts(o, d);
    for (int mu = 0; mu < d; mu++) {
        nn[mu] = n[mu];
        nb[mu] = max_blocks(static_cast<int>(n[mu]), shape_min_cut(d, mu, shape));
    }
    const bool g = gen && d >= 2;
    const bool one_solve = o.precision == TSYLV_FP64 || o.precision == TSYLV_DF64;
    size_t total = one_solve ? make_layout(d, nn, nb, g, 8, tab_ints_bound(d, nn, nb)).total
                             : make_ref_layout(d, nn, nb, g, tab_ints_bound(d, nn, nb)).total;
    if (o.host_io) {
        size_t N = 1, coef = 0;
        for (int mu = 0; mu < d; mu++) {
            N *= static_cast<size_t>(n[mu]);
            coef += static_cast<size_t>(n[mu]) * static_cast<size_t>(n[mu]);
        }
        total += ((gen ? 2 : 1) * coef + 2 * N) * sizeof(double) + 4 * 256;
    }
    return total;
}

size_t solver_residual_workspace_bytes(int d, const int64_t* n, bool gen) {
    if (!shape_ok(d, n)) return 0;
    long long nn[kMaxD];
    int nb[kMaxD];
    const int te = tile_extent(d);
    for (int mu = 0; mu < d; mu++) {
        nn[mu] = n[mu];
        nb[mu] = max_blocks(static_cast<int>(n[mu]), te);
    }
    return make_ref_layout(d, nn, nb, gen && d >= 2, tab_ints_bound(d, nn, nb)).total;
}

int solve_body(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
               void* work, size_t work_bytes, const tsylv_opts& o, int shape, tsylv_info* info, cudaStream_t stream,
               bool gen, bool transposed);
int solve_tuned(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
                void* work, size_t work_bytes, const tsylv_opts& o, tsylv_info* info, cudaStream_t stream, bool gen,
                bool transposed);

int solver_solve(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
                 void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream,
                 bool gen, bool transposed) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    const int sh = gen ? 1 : 0;  // argument numbers after A shift by one for the generalized form
    if (d < 1 || d > kMaxD) return -1;
    if (!shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    if (gen) {
        if (!C) return -4;
        for (int mu = 0; mu < d; mu++)
            if (!C[mu]) return -4;
    }
    if (!B) return -(4 + sh);
    if (!X) return -(5 + sh);
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -(6 + sh);
    if (work_bytes < solver_workspace_bytes(d, n, gen, o, transposed)) return -(7 + sh);
    if (int st = check_opts(o, d)) return st < 0 ? -(8 + sh) : st;
    // the tensor-core precisions run the persistent schedule only; the
    // generalized form is built for d <= 4
    if ((o.precision == TSYLV_TF32_REFINED || o.precision == TSYLV_BF16_REFINED) && o.schedule != 0)
        return TSYLV_EUNSUPPORTED;
    // the double-float solve: persistent schedule, d <= 4, FMA-style pair arithmetic
    if (o.precision == TSYLV_DF64 && (o.schedule != 0 || d > 4 || o.fp64_update == 2)) return TSYLV_EUNSUPPORTED;
    if (gen && d > 4) return TSYLV_EUNSUPPORTED;
    if (o.precision == TSYLV_FP64 && fp64_prod(o, d, o.schedule == 0) < 0) return TSYLV_EUNSUPPORTED;
    const int shape = shape_of_opts(o, d);
    if (shape >= 0) return solve_body(d, n, A, C, B, X, work, work_bytes, o, shape, info, stream, gen, transposed);
    return solve_tuned(d, n, A, C, B, X, work, work_bytes, o, info, stream, gen, transposed);
}

namespace {

// The autotuner of single solves (opts->nmin = -1): on the first call for a
// given order, mode sizes, form, direction and precision, every candidate
// tile shape (the leaf bound of every mode, shape_cut) solves the equation
// once, timed with CUDA events on `stream`; the fastest shape is kept for
// later calls.  The timing runs write X, never B: an in-place call (X == B)
// is not tuned and takes the default shape.
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tuned;

}  // namespace

int solve_tuned(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
                void* work, size_t work_bytes, const tsylv_opts& o, tsylv_info* info, cudaStream_t stream, bool gen,
                bool transposed) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<long long> key = {dev, d, gen ? 1 : 0, transposed ? 1 : 0, o.precision, o.schedule, o.partition,
                                  o.residual, o.fuse_step, o.resid_update, o.fp64_update};
    for (int mu = 0; mu < d; mu++) key.push_back(n[mu]);
    int shape = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) shape = it->second;
    }
    if (shape < 0 && static_cast<const void*>(X) == static_cast<const void*>(B)) shape = 0;
    if (shape < 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return cuda_fail_msg("autotuner events");
        }
        float best = 1e30f;
        int bs = 0;
        for (int s = 0; s < kShapes; s++) {
            if (d == 1 && s >= 4) break;  // shape 4 coincides with 3 for one mode
            float ms = 1e30f;
            for (int rep = 0; rep < 2; rep++) {  // the first run builds the plan and its graphs
                cudaEventRecord(e0, stream);
                const int st = solve_body(d, n, A, C, B, X, work, work_bytes, o, s, nullptr, stream, gen, transposed);
                cudaEventRecord(e1, stream);
                if (cudaEventSynchronize(e1) != cudaSuccess || st == TSYLV_ECUDA || st == TSYLV_ETIMEOUT) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st ? st : cuda_fail_msg("autotuner: synchronize");
                }
                if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 1e30f;
            }
            if (ms < best) {
                best = ms;
                bs = s;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        (void)cudaGetLastError();
        shape = bs;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = shape;
    }
    return solve_body(d, n, A, C, B, X, work, work_bytes, o, shape, info, stream, gen, transposed);
}

int solve_body(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B, double* X,
               void* work, size_t work_bytes, const tsylv_opts& o, int shape, tsylv_info* info, cudaStream_t stream,
               bool gen, bool transposed) {
    const int sh = gen ? 1 : 0;
    const bool df64 = o.precision == TSYLV_DF64;
    const bool refined = o.precision != TSYLV_FP64 && !df64;
    Call c;
    c.d = d;
    c.gen = gen && d >= 2;
    c.flip = transposed;
    c.df = o.residual == TSYLV_RESID_DF64;
    c.prod = o.precision == TSYLV_TF32_REFINED ? kProdTF32 : o.precision == TSYLV_BF16_REFINED ? kProdBF16 : kProdNative;
    if (!refined && !df64) {
        c.prod = fp64_prod(o, d, o.schedule == 0);
        if (c.prod < 0) return TSYLV_EUNSUPPORTED;
    }
    c.timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (int mu = 0; mu < d; mu++) {
        c.n[mu] = n[mu];
        c.A[mu] = A[mu];
        c.C[mu] = gen ? C[mu] : nullptr;
    }
    c.B = B;
    c.X = X;
    c.base = static_cast<char*>(work);
    (void)cudaGetLastError();  // launch checks below must not see errors of earlier, unrelated calls

    std::vector<uint8_t> sub;
    if (int st = read_structure(d, c.n, c.A, c.base, transposed, stream, sub)) return st;
    c.plan = get_plan(d, c.n, c.gen, refined ? 4 : 8, o.split, &sub, o.partition, shape);
    if (!c.plan) return cuda_fail_msg("plan: pinned host allocation");
    if (int st = prepare_kernels()) return st;
    c.timing = o.timing != 0;
    if (int st = ensure_events(c)) return st;
    c.persistent = o.schedule == 0;
    if (c.persistent) {
        if (df64) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
            const long long slots = static_cast<long long>(sms) * batched_occupancy_df(d, c.gen);
            c.flow_grid = static_cast<int>(c.plan->ntiles < slots ? c.plan->ntiles : slots);
        } else {
            c.flow_grid = flow_grid(refined ? 4 : 8, d, c.gen, c.plan->ntiles, c.prod);
        }
    }
    // pipelined first two steps: always (2), or by default (0) when the solve is
    // latency-bound, i.e. its largest wavefront has fewer than 5 blocks per SM
    // (measured: faster there, slower on wavefronts that fill the GPU)
    bool want_pipe = o.fuse_step == 2;
    if (o.fuse_step == 0 && refined && c.plan->n_rjobs > 0) {
        int wmax = 0;
        for (int w : c.plan->wave_cnt) wmax = std::max(wmax, w);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        want_pipe = wmax < 5 * sms;
    }
    c.pipe = refined && c.persistent && !c.gen && c.df && want_pipe && d >= 2 && c.plan->n_rjobs > 0 &&
             o.max_refine >= 2;
    if (c.pipe) c.pipe_grid = pipe_grid(d, 4 * c.plan->ntiles, c.prod);
    const int tagbase = (transposed ? 1 : 0) | (c.timing ? 2 : 0) | (c.df ? 4 : 0) | (c.persistent ? 256 : 0) |
                        (c.prod << 14) | (df64 ? 1 << 18 : 0);

    if (!refined) {
        c.L = make_layout(d, c.n, c.plan->nb, c.gen, 8, c.plan->tab.size());
        if (c.L.total > work_bytes) return -(7 + sh);
        int st = run_enqueue(*c.plan, make_key(c, tagbase), o.use_graph != 0, stream,
                             df64 ? enqueue_fp64_t<dfl> : enqueue_fp64_t<double>, c);
        if (st) return st;
        int herr = 0;
        if (cudaError_t e = cudaMemcpyAsync(&herr, c.base + c.L.err, sizeof(int), cudaMemcpyDeviceToHost, stream);
            e != cudaSuccess)
            return cuda_fail(e, "read status");
        if (cudaError_t e = cudaStreamSynchronize(stream); e != cudaSuccess)
            return cuda_fail(e, "synchronize after solve");
        if (info) {
            std::memset(info, 0, sizeof(*info));
            info->waves = static_cast<int>(c.plan->wave_off.size());
            info->launches = (c.persistent ? 2 : info->waves) + d * (c.gen ? 2 : 1) + 2;
            info->tiles = static_cast<int>(c.plan->ntiles);
            for (int mu = 0; mu < d; mu++) info->leaf[mu] = shape_cut(d, mu, shape);
            info->resid = -1;
            info->norm_A = -1;
            info->flops = c.plan->flops;
            if (c.timing) {
                float a = -1, b = -1;
                if (cudaEventElapsedTime(&a, c.plan->ev[0], c.plan->ev[3]) != cudaSuccess) a = -1;
                if (cudaEventElapsedTime(&b, c.plan->ev[1], c.plan->ev[2]) != cudaSuccess) b = -1;
                (void)cudaGetLastError();
                info->t_total_ms = a;
                info->t_waves_ms = b;
            }
        }
        return map_err(herr);
    }

    // ---- mixed-precision refinement
    c.R = make_ref_layout(d, c.n, c.plan->nb, c.gen, c.plan->tab.size());
    if (c.R.total > work_bytes) return -(7 + sh);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (c.timing) {
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaEventRecord(t0, stream);
    }
    int st = run_enqueue(*c.plan, make_key(c, tagbase | 16), o.use_graph != 0, stream, enqueue_ref_setup, c);
    if (st) return st;
    double hA[2 * kMaxD] = {}, hn[3] = {};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hn, c.base + c.R.nrm, 3 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read norms");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after set-up");
    double nA = -1;
    int iters = 0, status = TSYLV_ENOCONV;
    double rho = -1, t_resid = 0, t_waves = 0;
    if (!(hn[1] > 0)) {
        status = TSYLV_OK;  // B = 0: X = 0
        rho = 0;
    } else {
        double prev = HUGE_VAL;
        int stall = 0;
        for (int it = 0; it < std::max(1, o.max_refine); it++) {
            // from the second step on, once the correction is small, the
            // residual is updated from the FP32 correction instead of re-evaluated
            if (o.resid_update == 0 && it > 0 && prev <= 1e-5) c.update = true;
            c.first = it == 0;
            const bool pipe2 = c.pipe && it == 0;  // steps 1 and 2 in one launch
            st = run_enqueue(*c.plan,
                             make_key(c, tagbase | 32 | (pipe2 ? 4096 : (c.update ? 512 : 0) | (c.first ? 2048 : 0))),
                             o.use_graph != 0, stream, pipe2 ? enqueue_ref_pipe : enqueue_ref_iter, c);
            if (st) return st;
            if (pipe2) {
                // the first residual's norm decides, as for separate steps, whether
                // the second residual may be the FP32 update; if not, re-evaluate it
                double h1[3] = {}, hx[3] = {};
                if ((e = cudaMemcpyAsync(h1, c.base + c.R.nrm1, 3 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(hx, c.base + c.R.nrm, 3 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(hA, c.base + c.R.nA, 2 * kMaxD * 8, cudaMemcpyDeviceToHost, stream)) !=
                        cudaSuccess)
                    return cuda_fail(e, "read norms");
                if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize in refinement");
                nA = norm_op(c, hA);
                const double xn = std::sqrt(hx[2]);
                const double rho1 = (xn > 0 && nA > 0) ? std::sqrt(h1[0]) / (nA * xn) : 0.0;
                if (o.resid_update != 0 || !(rho1 <= 1e-5)) {
                    c.update = false;
                    c.first = false;
                    st = run_enqueue(*c.plan, make_key(c, tagbase | 8192), o.use_graph != 0, stream,
                                     enqueue_ref_resid_full, c);
                    if (st) return st;
                }
                prev = std::isfinite(rho1) ? rho1 : HUGE_VAL;
                c.update = false;
                it = 1;  // two steps done
            }
            if ((e = cudaMemcpyAsync(hn, c.base + c.R.nrm, 3 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
                return cuda_fail(e, "read residual norm");
            if (!c.update &&
                (e = cudaMemcpyAsync(hA, c.base + c.R.nA, 2 * kMaxD * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
                return cuda_fail(e, "read norms");
            if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize in refinement");
            if (!c.update) nA = norm_op(c, hA);
            iters = it + 1;
            if (c.timing) {
                float a = 0, b2 = 0;
                if (cudaEventElapsedTime(&a, c.plan->ev[1], c.plan->ev[2]) == cudaSuccess) t_resid += a;
                if (cudaEventElapsedTime(&b2, c.plan->ev[0], c.plan->ev[1]) == cudaSuccess) t_waves += b2;
                (void)cudaGetLastError();
            }
            const double xn = std::sqrt(hn[2]);
            rho = (xn > 0 && nA > 0) ? std::sqrt(hn[0]) / (nA * xn) : 0.0;
            if (!std::isfinite(rho)) {
                status = TSYLV_ENONFINITE;
                break;
            }
            if (rho <= o.tol) {
                status = TSYLV_OK;
                break;
            }
            if (rho > 0.5 * prev) {
                if (++stall >= 2) break;
            } else {
                stall = 0;
            }
            prev = rho;
        }
    }
    st = run_enqueue(*c.plan, make_key(c, tagbase | 64), o.use_graph != 0, stream, enqueue_ref_final, c);
    if (st) return st;
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, c.base + c.R.L32.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if (c.timing) cudaEventRecord(t1, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after refinement");
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = iters;
        info->waves = static_cast<int>(c.plan->wave_off.size());
        // separate steps: the solve (parameter store + launch, or one launch per
        // wavefront), the residual launches, scaling, update, reduction; the
        // pipelined first two steps: scaling, two parameter stores, one launch,
        // two updates, two reductions
        const int piped = c.pipe && iters >= 2 ? 2 : 0;
        info->launches = (iters - piped) * ((c.persistent ? 2 : info->waves) + (c.gen ? d : 1) + 4) +
                         (piped ? 8 : 0) + 4 * d + 8;
        info->tiles = static_cast<int>(c.plan->ntiles);
        for (int mu = 0; mu < d; mu++) info->leaf[mu] = shape_cut(d, mu, shape);
        info->resid = rho;
        info->norm_A = nA;
        info->flops = c.plan->flops * iters;
        if (c.timing) {
            float a = -1;
            if (cudaEventElapsedTime(&a, t0, t1) != cudaSuccess) a = -1;
            (void)cudaGetLastError();
            info->t_total_ms = a;
            info->t_resid_ms = t_resid;
            info->t_waves_ms = t_waves;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    const int ms = map_err(herr);
    if (ms == TSYLV_ETIMEOUT || ms == TSYLV_ECUDA) return ms;
    if (status == TSYLV_OK && ms == TSYLV_ESINGULAR) return ms;
    return status;
}

size_t solver_tt_workspace_bytes(int d, const int64_t* n, const tsylv_opts& o) {
    if (!shape_ok(d, n) || d < 2 || d > 4) return 0;
    long long nn[kMaxD];
    int nb[kMaxD];
    const int shape = shape_of_opts(o, d);
    for (int mu = 0; mu < d; mu++) {
        nn[mu] = n[mu];
        nb[mu] = max_blocks(static_cast<int>(n[mu]), shape_min_cut(d, mu, shape < 0 ? 0 : shape));
    }
    return make_layout(d, nn, nb, false, 8, tab_ints_bound(d, nn, nb), true).total;
}

// The paper's own generalized form Eq. (3.1): X x_1 A_1 + X x_1 C x_2 A_2
// ... x_d A_d = B, A_mu upper quasi-triangular, C upper triangular; the
// recursion of Sec. 3.1 as the block schedule of the other forms.  FP64,
// persistent schedule, d = 2..4.
int solver_solve_tt(int d, const int64_t* n, const double* const* A, const double* Cm, const double* B, double* X,
                    void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    if (d < 1 || d > kMaxD) return -1;
    if (!shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    if (!Cm) return -4;
    if (!B) return -5;
    if (!X) return -6;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -7;
    if (d < 2 || d > 4) return TSYLV_EUNSUPPORTED;
    if (work_bytes < solver_tt_workspace_bytes(d, n, o)) return -8;
    if (int st = check_opts(o, d)) return st < 0 ? -9 : st;
    const bool df64 = o.precision == TSYLV_DF64;
    if ((o.precision != TSYLV_FP64 && !df64) || o.schedule != 0 || o.nmin < 0 || o.fp64_update == 2)
        return TSYLV_EUNSUPPORTED;
    const int shape = shape_of_opts(o, d);
    Call c;
    c.d = d;
    c.gen = false;
    c.tt = true;
    c.timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (int mu = 0; mu < d; mu++) {
        c.n[mu] = n[mu];
        c.A[mu] = A[mu];
    }
    c.C[0] = Cm;
    c.B = B;
    c.X = X;
    c.base = static_cast<char*>(work);
    (void)cudaGetLastError();
    std::vector<uint8_t> sub;
    if (int st = read_structure(d, c.n, c.A, c.base, false, stream, sub)) return st;
    c.plan = get_plan(d, c.n, false, 8, o.split, &sub, o.partition, shape, true);
    if (!c.plan) return cuda_fail_msg("plan: pinned host allocation");
    if (int st = prepare_kernels()) return st;
    c.timing = o.timing != 0;
    if (int st = ensure_events(c)) return st;
    c.persistent = true;
    {
        static std::mutex m;
        static std::map<int, int> occ;
        int dev = 0;
        cudaGetDevice(&dev);
        int slots = 0;
        {
            std::lock_guard<std::mutex> lk(m);
            const int key = (dev * 8 + d) * 2 + (df64 ? 1 : 0);
            auto it = occ.find(key);
            if (it != occ.end()) {
                slots = it->second;
            } else {
                int sms = 0;
                if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
                slots = sms * (df64 ? batched_occupancy_tt_df(d) : batched_occupancy_tt(d));
                occ[key] = slots;
            }
        }
        c.flow_grid = static_cast<int>(c.plan->ntiles < slots ? c.plan->ntiles : slots);
    }
    c.L = make_layout(d, c.n, c.plan->nb, false, 8, c.plan->tab.size(), true);
    if (c.L.total > work_bytes) return -8;
    const int tag = 8192 * 4 | (c.timing ? 2 : 0) | (df64 ? 1 << 18 : 0);
    if (int st = run_enqueue(*c.plan, make_key(c, tag), o.use_graph != 0, stream,
                             df64 ? enqueue_tt_t<dfl> : enqueue_tt_t<double>, c))
        return st;
    int herr = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&herr, c.base + c.L.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after solve");
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->waves = static_cast<int>(c.plan->wave_off.size());
        info->launches = 2 + d + 1 + 2;
        info->tiles = static_cast<int>(c.plan->ntiles);
        for (int mu = 0; mu < d; mu++) info->leaf[mu] = shape_cut(d, mu, shape);
        info->resid = -1;
        info->norm_A = -1;
        info->flops = c.plan->flops;
        if (c.timing) {
            float a = -1, b = -1;
            if (cudaEventElapsedTime(&a, c.plan->ev[0], c.plan->ev[3]) != cudaSuccess) a = -1;
            if (cudaEventElapsedTime(&b, c.plan->ev[1], c.plan->ev[2]) != cudaSuccess) b = -1;
            (void)cudaGetLastError();
            info->t_total_ms = a;
            info->t_waves_ms = b;
        }
    }
    return map_err(herr);
}

size_t solver_z_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o) {
    if (!shape_ok(d, n) || d > 4) return 0;
    long long nn[kMaxD];
    int nb[kMaxD];
    const int shape = shape_of_opts(o, d);
    for (int mu = 0; mu < d; mu++) {
        nn[mu] = n[mu];
        nb[mu] = max_blocks(static_cast<int>(n[mu]), shape_min_cut(d, mu, shape < 0 ? 0 : shape));
    }
    return make_layout(d, nn, nb, gen && d >= 2, 16, tab_ints_bound(d, nn, nb)).total;
}

// The complex-triangular variant (Sec. 2.4: the coefficients reduced to
// complex Schur form, so every A_mu and C_mu is upper triangular and there are
// no coupled groups): the Laplace form Eq. (2.2) or the d-term form with
// complex FP64 coefficients and tensors (interleaved re, im); the same block
// partition, persistent schedule and base case as the real solves, in complex
// arithmetic.  d = 1..4, FP64, persistent schedule.
int solver_solve_z(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                   double* X, void* work, size_t work_bytes, const tsylv_opts* opts, tsylv_info* info,
                   cudaStream_t stream, bool gen) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    const int sh = gen ? 1 : 0;
    if (d < 1 || d > kMaxD) return -1;
    if (!shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    if (gen) {
        if (!C) return -4;
        for (int mu = 0; mu < d; mu++)
            if (!C[mu]) return -4;
    }
    if (!B) return -(4 + sh);
    if (!X) return -(5 + sh);
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -(6 + sh);
    if (d > 4) return TSYLV_EUNSUPPORTED;
    if (work_bytes < solver_z_workspace_bytes(d, n, gen, o)) return -(7 + sh);
    if (int st = check_opts(o, d)) return st < 0 ? -(8 + sh) : st;
    if (o.precision != TSYLV_FP64 || o.schedule != 0 || o.nmin < 0 || o.fp64_update == 2) return TSYLV_EUNSUPPORTED;
    const int shape = shape_of_opts(o, d);
    Call c;
    c.d = d;
    c.gen = gen && d >= 2;
    c.timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (int mu = 0; mu < d; mu++) {
        c.n[mu] = n[mu];
        c.A[mu] = A[mu];
        c.C[mu] = gen ? C[mu] : nullptr;
    }
    c.B = B;
    c.X = X;
    c.base = static_cast<char*>(work);
    (void)cudaGetLastError();
    // complex triangular coefficients: no 2x2 blocks, nothing to read back
    size_t nsub = 0;
    for (int mu = 0; mu < d; mu++) nsub += static_cast<size_t>(n[mu] - 1);
    std::vector<uint8_t> sub(nsub + 1, 0);
    c.plan = get_plan(d, c.n, c.gen, 16, o.split, &sub, o.partition, shape);
    if (!c.plan) return cuda_fail_msg("plan: pinned host allocation");
    if (int st = prepare_kernels()) return st;
    c.timing = o.timing != 0;
    if (int st = ensure_events(c)) return st;
    c.persistent = true;
    {
        static std::mutex m;
        static std::map<int, int> occ;
        int dev = 0;
        cudaGetDevice(&dev);
        const int key = (dev * 8 + d) * 2 + (c.gen ? 1 : 0);
        int slots = 0;
        {
            std::lock_guard<std::mutex> lk(m);
            auto it = occ.find(key);
            if (it != occ.end()) {
                slots = it->second;
            } else {
                int sms = 0;
                if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
                slots = sms * batched_occupancy_z(d, c.gen);
                occ[key] = slots;
            }
        }
        c.flow_grid = static_cast<int>(c.plan->ntiles < slots ? c.plan->ntiles : slots);
    }
    c.L = make_layout(d, c.n, c.plan->nb, c.gen, 16, c.plan->tab.size());
    if (c.L.total > work_bytes) return -(7 + sh);
    const int tag = 65536 | (c.timing ? 2 : 0);
    if (int st = run_enqueue(*c.plan, make_key(c, tag), o.use_graph != 0, stream, enqueue_z, c)) return st;
    int herr = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&herr, c.base + c.L.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after solve");
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->waves = static_cast<int>(c.plan->wave_off.size());
        info->launches = 2 + d * (c.gen ? 2 : 1) + 2;
        info->tiles = static_cast<int>(c.plan->ntiles);
        for (int mu = 0; mu < d; mu++) info->leaf[mu] = shape_cut(d, mu, shape);
        info->resid = -1;
        info->norm_A = -1;
        info->flops = 4.0 * c.plan->flops;  // a complex multiply-add is four real ones
        if (c.timing) {
            float a = -1, b = -1;
            if (cudaEventElapsedTime(&a, c.plan->ev[0], c.plan->ev[3]) != cudaSuccess) a = -1;
            if (cudaEventElapsedTime(&b, c.plan->ev[1], c.plan->ev[2]) != cudaSuccess) b = -1;
            (void)cudaGetLastError();
            info->t_total_ms = a;
            info->t_waves_ms = b;
        }
    }
    return map_err(herr);
}

// The failure path of the persistent schedule, exercised on purpose: the
// first block of a small solve is left out of the job queue, so the blocks
// that read it wait for a flag nothing sets until the bounded wait runs out.
int solver_selftest_wait_timeout(long long timeout_ns, cudaStream_t stream) {
    if (!(timeout_ns >= 1000000LL && timeout_ns <= 10000000000LL)) return -1;
    if (int st = prepare_kernels()) return st;
    const int d = 2;
    const long long n[2] = {32, 32};
    std::vector<uint8_t> sub(static_cast<size_t>(n[0] - 1 + n[1] - 1 + 1), 0);
    auto plan = get_plan(d, n, false, 8, 0, &sub, 0);
    if (!plan || plan->ntiles < 2) return cuda_fail_msg("self-test: plan");
    const Plan& p = *plan;
    const Layout L = make_layout(d, n, p.nb, false, 8, p.tab.size());
    void* mem = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&mem, L.total)) != cudaSuccess) return cuda_fail(e, "self-test: cudaMalloc");
    char* base = static_cast<char*>(mem);  // cudaMalloc memory is 256-byte aligned
    int herr = 0;
    auto run = [&]() -> cudaError_t {
        TRY(cudaMemsetAsync(base, 0, L.total, stream));  // zero coefficients and right-hand side
        TRY(cudaMemcpyAsync(base + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
        int* ctl = reinterpret_cast<int*>(base + L.fctl);
        WaveArgs wa = wave_args(p, L, base, timeout_ns);
        wa.ready = reinterpret_cast<int*>(base + L.flags);
        wa.abort = ctl + 1;
        wa.csize = 1;
        wa.timeout_ns = timeout_ns;
        WaveArgs* dargs = reinterpret_cast<WaveArgs*>(base + L.fargs);
        TRY(launch_store_args(wa, dargs, stream));
        BatchArgs ba{};
        ba.eqs = dargs;
        ba.jobs = nullptr;
        ba.tiles = reinterpret_cast<const int*>(base + L.tab) + p.t_wave + 1;  // the first block withheld
        ba.njobs = static_cast<int>(p.ntiles) - 1;
        ba.head = ctl;
        ba.abort = ctl + 1;
        ba.timeout_ns = timeout_ns;
        TRY(launch_batched<double>(d, false, ba, static_cast<int>(p.ntiles), stream));
        TRY(cudaMemcpyAsync(&herr, base + L.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
        return cudaStreamSynchronize(stream);
    };
    e = run();
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(e, "self-test: launch");
    return map_err(herr);
}

int solver_residual(int d, const int64_t* n, const double* const* A, const double* const* C, const double* B,
                    const double* X, double* R, double* rel, void* work, size_t work_bytes, const tsylv_opts* opts,
                    cudaStream_t stream) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    if (d < 1 || d > kMaxD) return -1;
    if (!shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    const bool gen = C != nullptr;
    if (gen)
        for (int mu = 0; mu < d; mu++)
            if (!C[mu]) return -4;
    if (!B) return -5;
    if (!X) return -6;
    if (!R) return -7;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -9;
    if (work_bytes < solver_residual_workspace_bytes(d, n, gen)) return -10;
    if (o.residual != TSYLV_RESID_DF64 && o.residual != TSYLV_RESID_FP64 || o.wait_ms < 1 || o.wait_ms > 600000)
        return -11;
    if (gen && d > 4) return TSYLV_EUNSUPPORTED;  // the generalized form is built for d <= 4
    Call c;
    c.d = d;
    c.gen = gen && d >= 2;
    c.df = o.residual == TSYLV_RESID_DF64;
    c.timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (int mu = 0; mu < d; mu++) {
        c.n[mu] = n[mu];
        c.A[mu] = A[mu];
        c.C[mu] = gen ? C[mu] : nullptr;
    }
    c.B = B;
    c.Xin = X;
    c.Rout = R;
    c.base = static_cast<char*>(work);
    (void)cudaGetLastError();
    std::vector<uint8_t> sub;
    if (int st = read_structure(d, c.n, c.A, c.base, false, stream, sub)) return st;
    c.plan = get_plan(d, c.n, c.gen, 4, 0, &sub, o.partition == 1 ? 1 : 0);
    if (!c.plan) return cuda_fail_msg("plan: pinned host allocation");
    if (int st = prepare_kernels()) return st;
    c.R = make_ref_layout(d, c.n, c.plan->nb, c.gen, c.plan->tab.size());
    if (c.R.total > work_bytes) return -10;
    int st = run_enqueue(*c.plan, make_key(c, (c.df ? 4 : 0) | 128), o.use_graph != 0, stream, enqueue_resid_api, c);
    if (st) return st;
    double hn[8] = {}, hA[2 * kMaxD] = {};
    int herr = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hn, c.base + c.R.nrm, 8 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hA, c.base + c.R.nA, 2 * kMaxD * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&herr, c.base + c.R.L32.err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "read residual norms");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "synchronize after residual");
    if (rel) {
        const double nA = norm_op(c, hA), xn = std::sqrt(hn[4]);
        *rel = (nA > 0 && xn > 0) ? std::sqrt(hn[0]) / (nA * xn) : 0.0;
    }
    return map_err(herr);
}

// Workspace of tsylv_backward: the transposed solve's workspace, then Lambda
// (N doubles, only when dB is not given -- sized unconditionally) and, for the
// generalized form, two N-double temporaries of the mode-product chains.
size_t solver_backward_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o) {
    const size_t ws = solver_workspace_bytes(d, n, gen, o, true);
    if (!ws) return 0;
    long long N = 1;
    for (int mu = 0; mu < d; mu++) N *= n[mu];
    return al256(ws) + al256(N * 8) * (gen ? 3 : 1);
}

int solver_backward(int d, const int64_t* n, const double* const* A, const double* const* C, const double* X,
                    const double* dX, double* dB, double* const* dA, double* const* dC, void* work, size_t work_bytes,
                    const tsylv_opts* opts, tsylv_info* info, cudaStream_t stream) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    if (d < 1 || d > kMaxD) return -1;
    if (!shape_ok(d, n)) return -2;
    if (!A) return -3;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -3;
    const bool gen = C != nullptr;
    if (gen)
        for (int mu = 0; mu < d; mu++)
            if (!C[mu]) return -4;
    if (!X) return -5;
    if (!dX) return -6;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -10;
    const size_t need = solver_backward_workspace_bytes(d, n, gen, o);
    if (!need || work_bytes < need) return -11;
    long long N = 1;
    for (int mu = 0; mu < d; mu++) N *= n[mu];
    const size_t ws = al256(solver_workspace_bytes(d, n, gen, o, true));
    char* base = static_cast<char*>(work);
    double* lam = dB ? dB : reinterpret_cast<double*>(base + ws);
    double* t0 = reinterpret_cast<double*>(base + ws + al256(N * 8));
    double* t1 = reinterpret_cast<double*>(base + ws + 2 * al256(N * 8));

    // Lambda = A^{-T}(dX): the transposed solve (index-flipped coefficients)
    tsylv_info si{};
    const int st = solver_solve(d, n, A, C, dX, lam, work, ws, &o, &si, stream, gen, true);
    if (st < 0) return st == -1 || st == -2 || st == -3 || st == -4 ? st : -11;
    if (st != TSYLV_OK && st != TSYLV_ENOCONV) return st;

    // X x_{eta in S} M_eta for the modes of S in increasing order; M_eta = A
    // for eta == special, else C.  Returns the pointer holding the result.
    int launches = 0;
    auto chain = [&](int skip, int special, const double** out) -> cudaError_t {
        const double* src = X;
        double* bufs[2] = {t0, t1};
        int which = 0;
        for (int eta = 0; eta < d; eta++) {
            if (eta == skip) continue;
            long long L = 1, R = 1;
            for (int q = 0; q < eta; q++) L *= n[q];
            for (int q = eta + 1; q < d; q++) R *= n[q];
            const bool isA = eta == special;
            const double* M = isA ? A[eta] : C[eta];
            cudaError_t e = launch_modeprod(src, M, bufs[which], L, static_cast<int>(n[eta]), R, isA, stream);
            if (e != cudaSuccess) return e;
            launches++;
            src = bufs[which];
            which ^= 1;
        }
        *out = src;
        return cudaSuccess;
    };

    for (int mu = 0; mu < d; mu++) {
        long long L = 1, R = 1;
        for (int q = 0; q < mu; q++) L *= n[q];
        for (int q = mu + 1; q < d; q++) R *= n[q];
        const int m = static_cast<int>(n[mu]);
        cudaError_t e;
        if (dA && dA[mu]) {
            const double* W = X;
            if (gen && d > 1 && (e = chain(mu, -1, &W)) != cudaSuccess) return cuda_fail(e, "backward: mode products");
            if ((e = cudaMemsetAsync(dA[mu], 0, sizeof(double) * m * m, stream)) != cudaSuccess)
                return cuda_fail(e, "backward: clear dA");
            if ((e = launch_gram(lam, W, dA[mu], L, m, R, stream)) != cudaSuccess)
                return cuda_fail(e, "backward: dA contraction");
            if ((e = launch_finalize_grad(dA[mu], A[mu], dA[mu], m, false, stream)) != cudaSuccess)
                return cuda_fail(e, "backward: dA mask");
            launches += 2;
        }
        if (gen && dC && dC[mu]) {
            if ((e = cudaMemsetAsync(dC[mu], 0, sizeof(double) * m * m, stream)) != cudaSuccess)
                return cuda_fail(e, "backward: clear dC");
            for (int nu = 0; nu < d; nu++) {
                if (nu == mu) continue;
                const double* W = nullptr;
                if ((e = chain(mu, nu, &W)) != cudaSuccess) return cuda_fail(e, "backward: mode products");
                if ((e = launch_gram(lam, W, dC[mu], L, m, R, stream)) != cudaSuccess)
                    return cuda_fail(e, "backward: dC contraction");
                launches++;
            }
            if ((e = launch_finalize_grad(dC[mu], C[mu], dC[mu], m, true, stream)) != cudaSuccess)
                return cuda_fail(e, "backward: dC mask");
            launches++;
        }
    }
    if (cudaError_t e = cudaStreamSynchronize(stream); e != cudaSuccess)
        return cuda_fail(e, "synchronize after backward");
    if (info) {
        *info = si;
        info->launches = si.launches + launches;
    }
    return st;
}

// ------------------------------------------------------------------ plans

struct SolvePlan {
    int d = 0;
    long long n[kMaxD] = {};
    const double* A[kMaxD] = {};
    const double* C[kMaxD] = {};
    bool gen = false, flip = false;
    int prod = kProdNative;
    int flow_grid = 0;
    bool use_graph = true;
    bool df64 = false;  // the double-float solve (TSYLV_DF64)
    long long timeout_ns = kTimeoutNs;
    std::shared_ptr<Plan> plan;
    Layout L;
    int dev = 0;
    uint8_t* pat = nullptr;  // device: A_mu(i + 1, i) != 0, modes back to back (unflipped)
};

int plan_create(void** out, int d, const int64_t* n, const double* const* A, const double* const* C, bool flip,
                void* work, size_t work_bytes, const tsylv_opts* opts, cudaStream_t stream) {
    if (!out) return -1;
    *out = nullptr;
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    const bool gen = C != nullptr;
    if (d < 1 || d > kMaxD) return -2;
    if (!shape_ok(d, n)) return -3;
    if (!A) return -4;
    for (int mu = 0; mu < d; mu++)
        if (!A[mu]) return -4;
    if (gen)
        for (int mu = 0; mu < d; mu++)
            if (!C[mu]) return -5;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -7;
    if (work_bytes < solver_workspace_bytes(d, n, gen, o, flip)) return -8;
    if (int st = check_opts(o, d)) return st < 0 ? -9 : st;
    const bool df64 = o.precision == TSYLV_DF64;
    if ((o.precision != TSYLV_FP64 && !df64) || o.nmin < 0 || o.timing || (gen && d > 4)) return TSYLV_EUNSUPPORTED;
    if (df64 && (o.schedule != 0 || d > 4 || o.fp64_update == 2)) return TSYLV_EUNSUPPORTED;
    const int prod = df64 ? kProdNative : fp64_prod(o, d, o.schedule == 0);
    if (prod < 0) return TSYLV_EUNSUPPORTED;
    (void)cudaGetLastError();
    auto sp = std::make_unique<SolvePlan>();
    sp->d = d;
    sp->gen = gen && d >= 2;
    sp->flip = flip;
    sp->prod = prod;
    sp->df64 = df64;
    sp->use_graph = o.use_graph != 0;
    sp->timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    for (int mu = 0; mu < d; mu++) {
        sp->n[mu] = n[mu];
        sp->A[mu] = A[mu];
        sp->C[mu] = gen ? C[mu] : nullptr;
    }
    std::vector<uint8_t> sub;
    if (int st = read_structure(d, sp->n, sp->A, static_cast<char*>(work), flip, stream, sub))
        return st == -3 ? -4 : st;
    sp->plan = get_plan(d, sp->n, sp->gen, 8, o.split, &sub, o.partition, shape_of_opts(o, d));
    if (!sp->plan) return cuda_fail_msg("plan: pinned host allocation");
    if (int st = prepare_kernels()) return st;
    if (o.schedule == 0) {
        if (df64) {
            int dv = 0, sms = 0;
            cudaGetDevice(&dv);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dv) != cudaSuccess || sms < 1) sms = 1;
            const long long slots = static_cast<long long>(sms) * batched_occupancy_df(d, sp->gen);
            sp->flow_grid = static_cast<int>(sp->plan->ntiles < slots ? sp->plan->ntiles : slots);
        } else {
            sp->flow_grid = flow_grid(8, d, sp->gen, sp->plan->ntiles, prod);
        }
    }
    sp->L = make_layout(d, sp->n, sp->plan->nb, sp->gen, 8, sp->plan->tab.size());
    if (sp->L.total > work_bytes) return -8;
    // the unflipped pattern, as the device check reads it
    size_t nsub = 0;
    for (int mu = 0; mu < d; mu++) nsub += static_cast<size_t>(n[mu] - 1);
    std::vector<uint8_t> raw(nsub + 1, 0);
    size_t off = 0;
    for (int mu = 0; mu < d; mu++) {
        const long long m = n[mu];
        for (long long i = 0; i + 1 < m; i++) raw[off + static_cast<size_t>(flip ? m - 2 - i : i)] = sub[off + i];
        off += static_cast<size_t>(m - 1);
    }
    cudaError_t e;
    if ((e = cudaGetDevice(&sp->dev)) != cudaSuccess) return cuda_fail(e, "plan: cudaGetDevice");
    if ((e = cudaMalloc(&sp->pat, raw.size())) != cudaSuccess) return cuda_fail(e, "plan: cudaMalloc");
    if ((e = cudaMemcpy(sp->pat, raw.data(), raw.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(sp->pat);
        return cuda_fail(e, "plan: structure upload");
    }
    *out = sp.release();
    return 0;
}

int plan_execute(void* handle, const double* B, double* X, void* work, size_t work_bytes, int* status,
                 cudaStream_t stream) {
    if (!handle) return -1;
    SolvePlan& sp = *static_cast<SolvePlan*>(handle);
    if (!B) return -2;
    if (!X) return -3;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -4;
    if (work_bytes < sp.L.total) return -5;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != sp.dev) return TSYLV_EUNSUPPORTED;
    (void)cudaGetLastError();
    Call c;
    c.d = sp.d;
    c.gen = sp.gen;
    c.flip = sp.flip;
    c.prod = sp.prod;
    c.timeout_ns = sp.timeout_ns;
    for (int mu = 0; mu < sp.d; mu++) {
        c.n[mu] = sp.n[mu];
        c.A[mu] = sp.A[mu];
        c.C[mu] = sp.C[mu];
    }
    c.B = B;
    c.X = X;
    c.base = static_cast<char*>(work);
    c.plan = sp.plan;
    c.L = sp.L;
    c.persistent = sp.flow_grid > 0;
    c.flow_grid = sp.flow_grid;
    c.pat = sp.pat;
    c.status_out = status;
    const int tag = (sp.flip ? 1 : 0) | (c.persistent ? 256 : 0) | (c.prod << 14) | (sp.df64 ? 1 << 18 : 0) | (1 << 20);
    return run_enqueue(*sp.plan, make_key(c, tag), sp.use_graph, stream,
                       sp.df64 ? enqueue_plan_t<dfl> : enqueue_plan_t<double>, c);
}

void plan_destroy(void* handle) {
    if (!handle) return;
    SolvePlan* sp = static_cast<SolvePlan*>(handle);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != sp->dev) cudaSetDevice(sp->dev);
    if (sp->pat) cudaFree(sp->pat);  // synchronises the device: no execution still reads the pattern
    if (cur != sp->dev) cudaSetDevice(cur);
    delete sp;
}

}  // namespace tsylv
