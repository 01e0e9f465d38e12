// Solve orchestration: structure read-back, schedule, graph capture/replay.
#include "solver.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "plan.h"

namespace tsylv {

namespace {

constexpr long long kTimeoutNs = 2000000000LL;  // bound of every device-side wait

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

// Upper bound of the block-table size for any admissible structure.
size_t tab_ints_bound(int d, const long long* n, const int* nb) {
    size_t t = 0, nt = 1;
    for (int mu = 0; mu < d; mu++) {
        t += 2 * static_cast<size_t>(nb[mu]) + static_cast<size_t>(n[mu]);
        nt *= static_cast<size_t>(nb[mu]);
    }
    return t + nt;
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

}  // namespace

size_t solver_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o, bool transposed) {
    (void)transposed;
    if (!shape_ok(d, n)) return 0;
    long long nn[kMaxD];
    int nb[kMaxD];
    const int te = tile_extent(d);
    for (int mu = 0; mu < d; mu++) {
        nn[mu] = n[mu];
        nb[mu] = max_blocks(static_cast<int>(n[mu]), te);
    }
    Layout L = make_layout(d, nn, nb, gen && d >= 2, 8, tab_ints_bound(d, nn, nb));
    size_t total = L.total;
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

namespace {

struct Call {
    int d = 0;
    bool gen = false, flip = false;
    long long n[kMaxD] = {};
    const double* A[kMaxD] = {};
    const double* C[kMaxD] = {};
    const double* B = nullptr;
    double* X = nullptr;
    char* base = nullptr;
    std::shared_ptr<Plan> plan;
    Layout L;
    bool timing = false;
};

inline cudaError_t mark(const Call& c, int i, cudaStream_t s) {
    // External: inside stream capture this becomes an event-record node of the graph
    return c.timing ? cudaEventRecordWithFlags(c.plan->ev[i], s, cudaEventRecordExternal) : cudaSuccess;
}

// Queue one FP64 solve of the planned block grid.
cudaError_t enqueue_fp64(const Call& c, cudaStream_t s) {
    const Plan& p = *c.plan;
    const Layout& L = c.L;
    char* base = c.base;
    GeomArgs g = geom_of(p, L, base, c.flip);
    cudaError_t e;
    if ((e = mark(c, 0, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(base + L.err, 0, 64, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(base + L.tab, p.h_tab, p.tab.size() * sizeof(int), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    for (int mu = 0; mu < p.d; mu++) {
        if ((e = launch_pack_coef<double>(g, mu, c.A[mu], reinterpret_cast<double*>(base + L.At[mu]), false, s)) !=
            cudaSuccess)
            return e;
        if (p.gen &&
            (e = launch_pack_coef<double>(g, mu, c.C[mu], reinterpret_cast<double*>(base + L.Ct[mu]), true, s)) !=
                cudaSuccess)
            return e;
    }
    double* Xt = reinterpret_cast<double*>(base + L.X);
    if ((e = launch_pack_tensor<double>(g, c.B, Xt, 1.0, s)) != cudaSuccess) return e;
    WaveArgs wa{};
    const int* tab = reinterpret_cast<const int*>(base + L.tab);
    for (int mu = 0; mu < p.d; mu++) {
        wa.nb[mu] = p.nb[mu];
        wa.hi[mu] = p.nb[mu];
        wa.tstride[mu] = p.tstride[mu];
        wa.bsize[mu] = tab + p.t_size[mu];
        wa.At[mu] = base + L.At[mu];
        wa.Ct[mu] = p.gen ? base + L.Ct[mu] : nullptr;
        wa.P[mu] = p.gen && mu >= 1 ? base + L.P[mu] : nullptr;
        wa.G[mu] = p.gen && mu >= 1 ? base + L.G[mu] : nullptr;
    }
    wa.X = Xt;
    wa.err = reinterpret_cast<int*>(base + L.err);
    wa.timeout_ns = kTimeoutNs;
    if ((e = mark(c, 1, s)) != cudaSuccess) return e;
    for (size_t w = 0; w < p.wave_off.size(); w++) {
        wa.tiles = tab + p.t_wave + p.wave_off[w];
        wa.ntiles = p.wave_cnt[w];
        wa.csize = p.wave_csize[w];
        if ((e = launch_wave<double>(p.d, p.gen, kProdNative, wa, s)) != cudaSuccess) return e;
    }
    if ((e = mark(c, 2, s)) != cudaSuccess) return e;
    if ((e = launch_unpack_tensor<double>(g, Xt, c.X, s)) != cudaSuccess) return e;
    return mark(c, 3, s);
}

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
            if (p.graphs.size() >= 16) {
                cudaGraphExecDestroy(p.graphs.front().exec);
                p.graphs.erase(p.graphs.begin());
            }
            p.graphs.push_back(GraphEntry{key, exec});
        }
    }
    if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return 0;
}

}  // namespace

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
    if (o.precision < TSYLV_FP64 || o.precision > TSYLV_BF16_REFINED || o.max_refine < 0 || !(o.tol > 0) ||
        (o.residual != TSYLV_RESID_DF64 && o.residual != TSYLV_RESID_FP64) || o.split < 0 || o.nmin < 0)
        return -(8 + sh);
    if (o.precision != TSYLV_FP64 || o.host_io || (o.nmin != 0 && o.nmin != tile_extent(d)))
        return TSYLV_EUNSUPPORTED;

    Call c;
    c.d = d;
    c.gen = gen && d >= 2;
    c.flip = transposed;
    for (int mu = 0; mu < d; mu++) {
        c.n[mu] = n[mu];
        c.A[mu] = A[mu];
        c.C[mu] = gen ? C[mu] : nullptr;
    }
    c.B = B;
    c.X = X;
    c.base = static_cast<char*>(work);

    (void)cudaGetLastError();  // launch checks below must not see errors of earlier, unrelated calls

    // 2x2 block structure: sub-diagonal of every A_mu, read back once per call
    size_t nsub = 0;
    for (int mu = 0; mu < d; mu++) nsub += static_cast<size_t>(n[mu] - 1);
    std::vector<double> hsub(nsub + 1, 0.0);
    {
        const size_t sub_off = 256;  // Layout::sub does not depend on the block counts
        double* dsub = reinterpret_cast<double*>(c.base + sub_off);
        if (nsub > 0) {
            cudaError_t e;
            if ((e = launch_gather_subdiag(d, c.n, c.A, dsub, stream)) != cudaSuccess)
                return cuda_fail(e, "gather sub-diagonal");
            if ((e = cudaMemcpyAsync(hsub.data(), dsub, nsub * sizeof(double), cudaMemcpyDeviceToHost, stream)) !=
                cudaSuccess)
                return cuda_fail(e, "read sub-diagonal");
        }
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "synchronize before planning");
    }
    std::vector<uint8_t> sub(nsub + 1, 0);
    {
        size_t off = 0;
        for (int mu = 0; mu < d; mu++) {
            const long long m = n[mu];
            for (long long i = 0; i + 1 < m; i++) {
                const size_t src = transposed ? off + static_cast<size_t>(m - 2 - i) : off + static_cast<size_t>(i);
                sub[off + i] = hsub[src] != 0.0 ? 1 : 0;
            }
            for (long long i = 0; i + 2 < m; i++)
                if (sub[off + i] && sub[off + i + 1]) return -3;  // not quasi-triangular
            off += static_cast<size_t>(m - 1);
        }
    }
    c.plan = get_plan(d, c.n, c.gen, 8, o.split, &sub);
    if (!c.plan) return cuda_fail_msg("plan: pinned host allocation");
    c.L = make_layout(d, c.n, c.plan->nb, c.gen, 8, c.plan->tab.size());
    if (c.L.total > work_bytes) return -(7 + sh);
    c.timing = o.timing != 0;
    if (c.timing && !c.plan->ev[0])
        for (auto& ev : c.plan->ev)
            if (cudaError_t e = cudaEventCreate(&ev); e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");

    {
        static std::mutex pm;
        static bool prepared[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(pm);
        if (dev >= 0 && dev < 64 && !prepared[dev]) {
            cudaError_t e = prepare_wave<double>();
            if (e == cudaSuccess) e = prepare_wave<float>();
            if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
            prepared[dev] = true;
        }
    }
    std::vector<const void*> key;
    for (int mu = 0; mu < d; mu++) {
        key.push_back(c.A[mu]);
        key.push_back(c.C[mu]);
    }
    key.push_back(B);
    key.push_back(X);
    key.push_back(work);
    key.push_back(reinterpret_cast<const void*>(static_cast<uintptr_t>((transposed ? 1 : 0) | (c.timing ? 2 : 0))));
    int st = run_enqueue(*c.plan, key, o.use_graph != 0, stream, enqueue_fp64, c);
    if (st) return st;
    int herr = 0;
    if (cudaError_t e = cudaMemcpyAsync(&herr, c.base + c.L.err, sizeof(int), cudaMemcpyDeviceToHost, stream);
        e != cudaSuccess)
        return cuda_fail(e, "read status");
    if (cudaError_t e = cudaStreamSynchronize(stream); e != cudaSuccess) return cuda_fail(e, "synchronize after solve");
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = 0;
        info->waves = static_cast<int>(c.plan->wave_off.size());
        info->launches = info->waves + d * (c.gen ? 2 : 1) + 2;
        info->tiles = static_cast<int>(c.plan->ntiles);
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

int solver_residual(int, const int64_t*, const double* const*, const double* const*, const double*, const double*,
                    double*, double*, void*, size_t, const tsylv_opts*, cudaStream_t) {
    return TSYLV_EUNSUPPORTED;
}

size_t solver_backward_workspace_bytes(int d, const int64_t* n, bool gen, const tsylv_opts& o) {
    return solver_workspace_bytes(d, n, gen, o, true);
}

int solver_backward(int, const int64_t*, const double* const*, const double* const*, const double*, const double*,
                    double*, double* const*, double* const*, void*, size_t, const tsylv_opts*, tsylv_info*,
                    cudaStream_t) {
    return TSYLV_EUNSUPPORTED;
}

size_t solver_batched_workspace_bytes(int, const int*, const int64_t*, bool, const tsylv_opts&) { return 0; }

int solver_batched(int, const int*, const int64_t*, const int64_t*, const int64_t*, const double*, const double*,
                   const double*, double*, void*, size_t, const tsylv_opts*, int*, tsylv_info*, cudaStream_t) {
    return TSYLV_EUNSUPPORTED;
}

}  // namespace tsylv
