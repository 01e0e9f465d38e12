// Host driver of tsylv_solve_batched: per-equation block partitions (the
// split rule of Alg. 2 applied to each mode, exactly as for one solve), the
// job queue of the persistent launch, a small autotuner for the launch
// (queue order and resident CTAs per SM), and the captured CUDA graph
// (control reset, table upload, packing, the persistent launch per order d,
// unpacking, status read-back).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

#include "apply_kernel.cuh"
#include "batched.h"
#include "plan.h"
#include "refine.h"
#include "solver.h"

namespace tsylv {

namespace {

// bound of every device-side wait of the current call (opts->wait_ms), set
// at the start of each call on the calling thread
thread_local long long t_timeout_ns = 2000000000LL;
constexpr int kPolicies = 3;  // 0: longest remaining path first, 1: wavefront-major, 2: equation-major

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

struct EqPlan {
    int d = 0;
    long long n[kMaxD] = {};
    Part part[kMaxD];
    int nb[kMaxD] = {};
    long long tstride[kMaxD] = {};
    long long ntiles = 0;
    int nwaves = 0;
    // workspace offsets (bytes, from the data region)
    size_t X = 0, P[kMaxD] = {}, G[kMaxD] = {}, At[kMaxD] = {}, Ct[kMaxD] = {};
    size_t part_off[kMaxD] = {};  // ints in the table: start (nb), then size (nb)
    size_t flag_off = 0;          // first "solved" flag of this equation's blocks
};

struct BatchGraph {
    std::vector<const void*> key;
    cudaGraphExec_t exec = nullptr;
};

struct BatchPlan {
    int count = 0;
    bool gen = false;
    std::vector<EqPlan> eq;
    std::vector<int> dlist;                 // distinct orders, increasing
    std::vector<BatchJob> jobs[kPolicies];  // per policy; segments by order d
    std::vector<int> seg_off, seg_cnt;      // per entry of dlist (same for every policy)
    std::vector<BatchCoefJob> cjobs;
    size_t data_bytes = 0;
    std::vector<long long> tile_off;        // first global block of every equation (count + 1 entries)
    double flops = 0;
    int tuned_policy = -1, tuned_grid = 0, tuned_shape = 0;  // autotuner result (kept on the default-shape plan)
    std::vector<BatchGraph> graphs;
    ~BatchPlan() {
        for (auto& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    }
};

// Regions of the batched workspace (byte offsets from its base).
struct BatchLayout {
    size_t ctl = 0;    // heads [4], abort, pad [3], done [count], errs [count]
    size_t flags = 0;  // per-block "solved" flags of every equation
    size_t sub = 0;    // sub-diagonals of every A_mu, then the gather tables
    size_t tab = 0;    // WaveArgs [count], BatchGeom [count], jobs, coefficient jobs, partition ints
    size_t data = 0;   // block tensors and coefficient tiles
    size_t total = 0;
    size_t o_wave = 0, o_geom = 0, o_jobs = 0, o_cjobs = 0, o_part = 0, tab_bytes = 0;
    size_t o_aoff = 0, o_nmat = 0, o_ooff = 0, nsub = 0;
};

// Upper bounds of one equation's block counts and data bytes (any admissible
// structure), region by region as get_batch_plan lays them out.
void eq_bounds(int d, const int64_t* n, bool gen, int elem, int shape, long long& tiles, long long& ctiles,
               long long& pints, size_t& data) {
    const int te = tile_extent(d);
    const size_t td = static_cast<size_t>(ipow(te, d)), tc = static_cast<size_t>(te) * te;
    const bool g = gen && d >= 2;
    tiles = 1;
    ctiles = 0;
    pints = 0;
    data = 0;
    for (int mu = 0; mu < d; mu++) {
        const long long nb = max_blocks(static_cast<int>(n[mu]), shape_min_cut(d, mu, shape));
        tiles *= nb;
        ctiles += nb * (nb + 1) / 2;
        pints += 2 * nb;
        data += (g ? 2 : 1) * al256(static_cast<size_t>(nb * (nb + 1) / 2) * tc * elem);
    }
    data += (g ? 1 + 2 * (d - 1) : 1) * al256(static_cast<size_t>(tiles) * td * elem);
}

BatchLayout make_batch_layout(int count, const int* d, const int64_t* n_packed, bool gen, int elem,
                              long long njobs, long long ncjobs, long long pints, size_t data_bytes) {
    BatchLayout L;
    size_t off = 0;
    L.ctl = off;
    off += al256((8 + 2 * static_cast<size_t>(count)) * sizeof(int));
    L.flags = off;
    off += al256(static_cast<size_t>(njobs) * sizeof(int));
    size_t nsub = 0, nmats = 0, k = 0;
    for (int e = 0; e < count; e++)
        for (int mu = 0; mu < d[e]; mu++, k++) {
            nsub += static_cast<size_t>(n_packed[k] > 0 ? n_packed[k] - 1 : 0);
            nmats++;
        }
    L.nsub = nsub;
    L.sub = off;
    off += al256((nsub + 1) * sizeof(double));
    L.o_aoff = off;
    off += al256(nmats * sizeof(long long));
    L.o_nmat = off;
    off += al256(nmats * sizeof(long long));
    L.o_ooff = off;
    off += al256(nmats * sizeof(long long));
    L.tab = off;
    size_t t = 0;
    L.o_wave = t;
    t += al256(count * sizeof(WaveArgs));
    L.o_geom = t;
    t += al256(count * sizeof(BatchGeom));
    L.o_jobs = t;
    t += al256(njobs * sizeof(BatchJob));
    L.o_cjobs = t;
    t += al256(ncjobs * sizeof(BatchCoefJob));
    L.o_part = t;
    t += al256(pints * sizeof(int));
    L.tab_bytes = t;
    off += t;
    L.data = off;
    off += data_bytes;
    L.total = off;
    (void)gen;
    (void)elem;
    return L;
}

struct Bounds {
    long long jobs = 0, cjobs = 0, pints = 0;
    size_t data = 0;
};

// shape: the tile shape the call uses (-1: any candidate of the autotuner)
Bounds batch_bounds(int count, const int* d, const int64_t* n_packed, bool gen, int elem, int shape) {
    Bounds b;
    size_t k = 0;
    for (int e = 0; e < count; e++) {
        long long t, c, p;
        size_t db;
        eq_bounds(d[e], n_packed + k, gen, elem, shape, t, c, p, db);
        b.jobs += t;
        b.cjobs += c;
        b.pints += p;
        b.data += db;
        k += static_cast<size_t>(d[e]);
    }
    return b;
}

bool shapes_ok(int count, const int* d, const int64_t* n_packed) {
    if (count < 1 || !d || !n_packed) return false;
    size_t k = 0;
    for (int e = 0; e < count; e++) {
        if (d[e] < 1 || d[e] > kMaxD) return false;
        long long N = 1;
        for (int mu = 0; mu < d[e]; mu++, k++) {
            if (n_packed[k] < 1 || n_packed[k] > (1LL << 30)) return false;
            N *= n_packed[k];
            if (N > (1LL << 40)) return false;
        }
    }
    return true;
}

std::mutex g_bmu;
std::map<std::vector<long long>, std::shared_ptr<BatchPlan>> g_bplans;

// Queue order of the jobs of one order-d segment under a policy.  Every
// order keeps each equation's wavefronts increasing, so a job's prerequisites
// always sit earlier in the queue.
void order_jobs(const BatchPlan& p, const std::vector<int>& eqs, int policy, std::vector<BatchJob>& out) {
    struct Item {
        int eq, tile, wave, need;
    };
    std::vector<Item> items;
    for (int e : eqs) {
        const EqPlan& q = p.eq[e];
        std::vector<std::vector<int>> waves(static_cast<size_t>(q.nwaves));
        for (long long t = 0; t < q.ntiles; t++) {
            int w = 0;
            for (int mu = 0; mu < q.d; mu++) w += q.nb[mu] - 1 - static_cast<int>((t / q.tstride[mu]) % q.nb[mu]);
            waves[static_cast<size_t>(w)].push_back(static_cast<int>(t));
        }
        int before = 0;
        for (int w = 0; w < q.nwaves; w++) {
            for (int t : waves[static_cast<size_t>(w)]) items.push_back({e, t, w, before});
            before += static_cast<int>(waves[static_cast<size_t>(w)].size());
        }
    }
    auto rem = [&](const Item& it) { return p.eq[it.eq].nwaves - 1 - it.wave; };
    if (policy == 0) {
        std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
            if (rem(a) != rem(b)) return rem(a) > rem(b);
            return a.eq < b.eq;
        });
    } else if (policy == 1) {
        std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
            if (a.wave != b.wave) return a.wave < b.wave;
            return a.eq < b.eq;
        });
    } else {
        std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
            const long long wa = p.eq[a.eq].ntiles, wb = p.eq[b.eq].ntiles;
            if (wa != wb) return wa > wb;
            if (a.eq != b.eq) return a.eq < b.eq;
            return a.wave < b.wave;
        });
    }
    // every job waits per source block on its "solved" flag, so no count is needed
    for (const Item& it : items) out.push_back({it.eq, it.tile, 0, 0});
}

double eq_flops(const EqPlan& q, bool gen) {
    // executed flops of the block updates (dense TE-tiles) and the base cases
    const int te = tile_extent(q.d);
    const double td = std::pow(te, q.d);
    double f = 0;
    for (long long t = 0; t < q.ntiles; t++) {
        for (int mu = 0; mu < q.d; mu++) {
            const int I = static_cast<int>((t / q.tstride[mu]) % q.nb[mu]);
            const double srcs = q.nb[mu] - 1 - I;
            f += srcs * 2.0 * td * te * (gen && q.d >= 2 ? 2.0 : 1.0);
        }
        f += td * (2.0 * q.d * te + 1);
    }
    return f;
}

std::shared_ptr<BatchPlan> get_batch_plan(int count, const int* d, const int64_t* n_packed, bool gen, int elem,
                                          const std::vector<uint8_t>& sub, int partition, int shape,
                                          int variant = 0) {
    // variant 1: the double-float batch (same layout as FP64; own tuning and graphs)
    std::vector<long long> key = {count, gen ? 1 : 0, elem, partition, shape, variant};
    size_t k = 0;
    for (int e = 0; e < count; e++) {
        key.push_back(d[e]);
        for (int mu = 0; mu < d[e]; mu++, k++) key.push_back(n_packed[k]);
    }
    // structure bits, packed 60 per word
    long long word = 0;
    int bits = 0;
    for (uint8_t s : sub) {
        word |= static_cast<long long>(s & 1) << bits;
        if (++bits == 60) {
            key.push_back(word);
            word = 0;
            bits = 0;
        }
    }
    key.push_back(word);
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bplans.find(key);
    if (it != g_bplans.end()) return it->second;
    if (g_bplans.size() > 64) g_bplans.clear();
    auto p = std::make_shared<BatchPlan>();
    p->count = count;
    p->gen = gen;
    p->eq.resize(count);
    k = 0;
    size_t soff = 0, data = 0, pints = 0, flags = 0;
    for (int e = 0; e < count; e++) {
        EqPlan& q = p->eq[e];
        q.d = d[e];
        const int te = tile_extent(q.d);
        long long ts = 1;
        int nw = 1;
        for (int mu = 0; mu < q.d; mu++, k++) {
            q.n[mu] = n_packed[k];
            std::vector<uint8_t> s(sub.begin() + static_cast<long long>(soff),
                                   sub.begin() + static_cast<long long>(soff + q.n[mu] - 1));
            soff += static_cast<size_t>(q.n[mu] - 1);
            q.part[mu] = make_part(static_cast<int>(q.n[mu]), s, shape_cut(q.d, mu, shape), partition);
            q.nb[mu] = q.part[mu].nb;
            q.tstride[mu] = ts;
            ts *= q.nb[mu];
            nw += q.nb[mu] - 1;
            q.part_off[mu] = pints;
            pints += 2 * static_cast<size_t>(q.nb[mu]);
        }
        q.ntiles = ts;
        q.nwaves = nw;
        q.flag_off = flags;
        flags += static_cast<size_t>(ts);
        const size_t td = static_cast<size_t>(ipow(te, q.d)), tc = static_cast<size_t>(te) * te;
        const bool g = gen && q.d >= 2;
        if (g)
            for (int l = 1; l < q.d; l++) {
                q.P[l] = data;
                data += al256(q.ntiles * td * elem);
                q.G[l] = data;
                data += al256(q.ntiles * td * elem);
            }
        for (int mu = 0; mu < q.d; mu++) {
            const size_t nct = static_cast<size_t>(q.nb[mu]) * (q.nb[mu] + 1) / 2;
            q.At[mu] = data;
            data += al256(nct * tc * elem);
            if (g) {
                q.Ct[mu] = data;
                data += al256(nct * tc * elem);
            }
            for (int J = 0; J < q.nb[mu]; J++)
                for (int I = 0; I <= J; I++) p->cjobs.push_back({e, mu, I, J});
        }
        p->flops += eq_flops(q, gen);
    }
    // the block tensors of all equations form one pool, in equation order, one
    // block after the other (pooled elementwise kernels index it by global block)
    p->tile_off.assign(static_cast<size_t>(count) + 1, 0);
    for (int e = 0; e < count; e++) {
        EqPlan& q = p->eq[e];
        const size_t td = static_cast<size_t>(ipow(tile_extent(q.d), q.d));
        p->tile_off[e + 1] = p->tile_off[e] + q.ntiles;
        q.X = data;
        data += q.ntiles * td * elem;
    }
    data = al256(data);
    p->data_bytes = data;
    for (int e = 0; e < count; e++)
        if (std::find(p->dlist.begin(), p->dlist.end(), d[e]) == p->dlist.end()) p->dlist.push_back(d[e]);
    std::sort(p->dlist.begin(), p->dlist.end());
    for (int pol = 0; pol < kPolicies; pol++) {
        for (int dd : p->dlist) {
            std::vector<int> eqs;
            for (int e = 0; e < count; e++)
                if (d[e] == dd) eqs.push_back(e);
            if (pol == 0) p->seg_off.push_back(static_cast<int>(p->jobs[pol].size()));
            order_jobs(*p, eqs, pol, p->jobs[pol]);
            if (pol == 0) p->seg_cnt.push_back(static_cast<int>(p->jobs[pol].size()) - p->seg_off.back());
        }
    }
    g_bplans[key] = p;
    return p;
}

// Layout of one plan with its own table and data sizes (within the bounds'
// layout the workspace was sized for): the table uploaded per call is then no
// larger than the plan needs.
BatchLayout plan_layout(const BatchPlan& p, const int* d, const int64_t* n_packed, int elem) {
    long long pints = 0;
    for (const EqPlan& q : p.eq)
        for (int mu = 0; mu < q.d; mu++) pints += 2 * q.nb[mu];
    return make_batch_layout(p.count, d, n_packed, p.gen, elem, static_cast<long long>(p.jobs[0].size()),
                             static_cast<long long>(p.cjobs.size()), pints, p.data_bytes);
}

// The uploaded table of one call: parameter blocks with device pointers into
// this workspace, the job lists and the partitions.
void fill_table(const BatchPlan& p, const BatchLayout& L, char* base, int policy, std::vector<unsigned char>& out,
                const int64_t* off_A, const int64_t* off_X) {
    out.assign(L.tab_bytes, 0);
    char* dev_tab = base + L.tab;
    char* dev_data = base + L.data;
    int* errs = reinterpret_cast<int*>(base + L.ctl) + 8 + p.count;
    const int* dev_part = reinterpret_cast<const int*>(dev_tab + L.o_part);
    int* hpart = reinterpret_cast<int*>(out.data() + L.o_part);
    WaveArgs* hw = reinterpret_cast<WaveArgs*>(out.data() + L.o_wave);
    BatchGeom* hg = reinterpret_cast<BatchGeom*>(out.data() + L.o_geom);
    size_t k = 0;
    for (int e = 0; e < p.count; e++) {
        const EqPlan& q = p.eq[e];
        const bool g = p.gen && q.d >= 2;
        WaveArgs wa{};
        BatchGeom ge{};
        ge.d = q.d;
        ge.xoff = off_X[e];
        for (int mu = 0; mu < q.d; mu++, k++) {
            std::memcpy(hpart + q.part_off[mu], q.part[mu].start.data(), sizeof(int) * q.nb[mu]);
            std::memcpy(hpart + q.part_off[mu] + q.nb[mu], q.part[mu].size.data(), sizeof(int) * q.nb[mu]);
            wa.nb[mu] = q.nb[mu];
            wa.hi[mu] = q.nb[mu];
            wa.tstride[mu] = q.tstride[mu];
            wa.bsize[mu] = dev_part + q.part_off[mu] + q.nb[mu];
            wa.At[mu] = dev_data + q.At[mu];
            wa.Ct[mu] = g ? dev_data + q.Ct[mu] : nullptr;
            wa.P[mu] = g && mu >= 1 ? dev_data + q.P[mu] : nullptr;
            wa.G[mu] = g && mu >= 1 ? dev_data + q.G[mu] : nullptr;
            ge.nb[mu] = q.nb[mu];
            ge.n[mu] = q.n[mu];
            ge.tstride[mu] = q.tstride[mu];
            ge.start[mu] = dev_part + q.part_off[mu];
            ge.size[mu] = dev_part + q.part_off[mu] + q.nb[mu];
            ge.aoff[mu] = off_A[k];
            ge.At[mu] = dev_data + q.At[mu];
            ge.Ct[mu] = g ? dev_data + q.Ct[mu] : nullptr;
        }
        wa.tiles = nullptr;
        wa.ntiles = static_cast<int>(q.ntiles);
        wa.csize = 1;
        wa.X = dev_data + q.X;
        wa.err = errs + e;
        wa.timeout_ns = t_timeout_ns;
        wa.ready = reinterpret_cast<const int*>(base + L.flags) + q.flag_off;
        wa.abort = reinterpret_cast<int*>(base + L.ctl) + 4;
        ge.X = dev_data + q.X;
        hw[e] = wa;
        hg[e] = ge;
    }
    std::memcpy(out.data() + L.o_jobs, p.jobs[policy].data(), p.jobs[policy].size() * sizeof(BatchJob));
    std::memcpy(out.data() + L.o_cjobs, p.cjobs.data(), p.cjobs.size() * sizeof(BatchCoefJob));
}

struct Pinned {
    unsigned char* ptr = nullptr;
    size_t bytes = 0;
    ~Pinned() {
        if (ptr) cudaFreeHost(ptr);
    }
    bool reserve(size_t b) {
        if (b <= bytes) return true;
        if (ptr) cudaFreeHost(ptr);
        ptr = nullptr;
        bytes = 0;
        if (cudaMallocHost(&ptr, b) != cudaSuccess) return false;
        bytes = b;
        return true;
    }
};

// Pinned staging of the host tables (per thread: calls on one thread are ordered
// by their synchronisation at the end).
thread_local Pinned t_pin_tab, t_pin_small;

int occupancy_cached(int d, bool gen, int elem = 8, bool df64 = false) {
    static std::mutex m;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const int key = ((dev * 16 + d * 2 + (gen ? 1 : 0)) * 2 + (elem == 4 ? 1 : 0)) * 2 + (df64 ? 1 : 0);
    std::lock_guard<std::mutex> lk(m);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int o = elem == 4 ? batched_occupancy<float>(d, gen)
                            : df64 ? batched_occupancy_df(d, gen) : batched_occupancy<double>(d, gen);
    cache[key] = o;
    return o;
}

int sm_count() {
    static int sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        sms[dev] = v;
    }
    return sms[dev];
}

int prepare_batched_once() {
    static std::mutex pm;
    static bool prepared[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(pm);
    if (dev >= 0 && dev < 64 && !prepared[dev]) {
        cudaError_t e = prepare_batched<double>();
        if (e == cudaSuccess) e = prepare_batched<float>();
        if (e == cudaSuccess) e = prepare_apply_batched();
        if (e != cudaSuccess) return cuda_fail(e, "batched kernel attributes");
        prepared[dev] = true;
    }
    return 0;
}

struct BatchCall {
    const BatchPlan* plan = nullptr;
    BatchLayout L;
    char* base = nullptr;
    const unsigned char* htab = nullptr;
    const double *A = nullptr, *C = nullptr, *B = nullptr;
    double* X = nullptr;
    int grid_per_sm[kMaxD + 1] = {};
    int* herr = nullptr;   // pinned host copy of the per-equation status words
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the persistent launches (autotuner)
    bool unpack = true;    // false for the autotuner's timing runs: X may alias B
    bool df64 = false;     // the double-float solve (pairs of floats in the block tensors)
};

cudaError_t enqueue_batch(const BatchCall& c, cudaStream_t s) {
    const BatchPlan& p = *c.plan;
    int* ctl = reinterpret_cast<int*>(c.base + c.L.ctl);
    char* tab = c.base + c.L.tab;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctl, 0, (8 + 2 * static_cast<size_t>(p.count)) * sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c.base + c.L.flags, 0, p.jobs[0].size() * sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(tab, c.htab, c.L.tab_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    const BatchGeom* geo = reinterpret_cast<const BatchGeom*>(tab + c.L.o_geom);
    const BatchJob* jobs = reinterpret_cast<const BatchJob*>(tab + c.L.o_jobs);
    const BatchCoefJob* cjobs = reinterpret_cast<const BatchCoefJob*>(tab + c.L.o_cjobs);
    const int njobs = static_cast<int>(p.jobs[0].size());
    if ((e = c.df64 ? launch_batch_pack<dfl>(geo, jobs, njobs, cjobs, static_cast<int>(p.cjobs.size()), c.B, c.A,
                                             p.gen ? c.C : nullptr, s)
                    : launch_batch_pack<double>(geo, jobs, njobs, cjobs, static_cast<int>(p.cjobs.size()), c.B, c.A,
                                                p.gen ? c.C : nullptr, s)) != cudaSuccess)
        return e;
    if (c.ev0 && (e = cudaEventRecord(c.ev0, s)) != cudaSuccess) return e;
    for (size_t g = 0; g < p.dlist.size(); g++) {
        BatchArgs a{};
        a.eqs = reinterpret_cast<const WaveArgs*>(tab + c.L.o_wave);
        a.jobs = jobs + p.seg_off[g];
        a.njobs = p.seg_cnt[g];
        a.head = ctl + g;
        a.abort = ctl + 4;
        a.done = ctl + 8;
        a.timeout_ns = t_timeout_ns;
        const int dd = p.dlist[g];
        int grid = c.grid_per_sm[dd] * sm_count();
        if (grid > a.njobs) grid = a.njobs;
        if (grid < 1) grid = 1;
        if ((e = c.df64 ? launch_batched_df(dd, p.gen, a, grid, s) : launch_batched<double>(dd, p.gen, a, grid, s)) !=
            cudaSuccess)
            return e;
    }
    if (c.ev1 && (e = cudaEventRecord(c.ev1, s)) != cudaSuccess) return e;
    if (c.unpack && (e = c.df64 ? launch_batch_unpack<dfl>(geo, jobs, njobs, c.X, s)
                                : launch_batch_unpack<double>(geo, jobs, njobs, c.X, s)) != cudaSuccess)
        return e;
    return cudaMemcpyAsync(c.herr, ctl + 8 + p.count, sizeof(int) * p.count, cudaMemcpyDeviceToHost, s);
}

// Capture (once per key) and launch a CUDA graph of `fn`, or run it eagerly.
int run_graph(BatchPlan& plan, const std::vector<const void*>& key, bool use_graph, cudaStream_t stream,
              const std::function<cudaError_t(cudaStream_t)>& fn, const char* what) {
    cudaError_t e;
    if (!use_graph) {
        if ((e = fn(stream)) != cudaSuccess) return cuda_fail(e, what);
        return 0;
    }
    cudaGraphExec_t exec = nullptr;
    for (auto& g : plan.graphs)
        if (g.key == key) exec = g.exec;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = capture_stream();
        if (!cs) return cuda_fail_msg("batched: capture stream");
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "batched: begin capture");
        const cudaError_t ee = fn(cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ee, what);
        }
        if (e != cudaSuccess) return cuda_fail(e, "batched: end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "batched: instantiate");
        if (plan.graphs.size() >= 16) {
            cudaGraphExecDestroy(plan.graphs.front().exec);
            plan.graphs.erase(plan.graphs.begin());
        }
        plan.graphs.push_back({key, exec});
    }
    if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return cuda_fail(e, "batched: graph launch");
    return 0;
}

// Same precedence as a single solve.
int map_status(int e) {
    if (e & kErrBounds) return cuda_fail_msg("device self-check: index outside a block array");
    if (e & kErrTimeout) return TSYLV_ETIMEOUT;
    if (e & kErrSingular) return TSYLV_ESINGULAR;
    if (e & kErrNonfinite) return TSYLV_ENONFINITE;
    return TSYLV_OK;
}

// The 2x2 structure of every A_mu (sub-diagonals gathered in one launch and
// read back), validated; herr receives pinned room for the status words.
int batch_structure(int count, const int* d, const int64_t* n_packed, const int64_t* off_A, const double* A_pool,
                    char* base, const BatchLayout& L, int* per_status, cudaStream_t stream, std::vector<uint8_t>& sub,
                    int*& herr) {
    size_t nmats = 0;
    for (int e = 0; e < count; e++) nmats += static_cast<size_t>(d[e]);
    std::vector<long long> aoff(nmats), nmat(nmats), ooff(nmats);
    long long maxn = 1;
    {
        size_t k = 0, so = 0;
        for (int e = 0; e < count; e++)
            for (int mu = 0; mu < d[e]; mu++, k++) {
                aoff[k] = off_A[k];
                nmat[k] = n_packed[k];
                ooff[k] = static_cast<long long>(so);
                so += static_cast<size_t>(n_packed[k] - 1);
                maxn = std::max<long long>(maxn, n_packed[k]);
            }
    }
    const size_t small_bytes = 3 * nmats * sizeof(long long) + (L.nsub + 1) * sizeof(double) + count * sizeof(int);
    if (!t_pin_small.reserve(small_bytes)) return cuda_fail_msg("batched: pinned host allocation");
    long long* hoffs = reinterpret_cast<long long*>(t_pin_small.ptr);
    double* hsub = reinterpret_cast<double*>(t_pin_small.ptr + 3 * nmats * sizeof(long long));
    herr = reinterpret_cast<int*>(t_pin_small.ptr + 3 * nmats * sizeof(long long) + (L.nsub + 1) * sizeof(double));
    std::memcpy(hoffs, aoff.data(), nmats * sizeof(long long));
    std::memcpy(hoffs + nmats, nmat.data(), nmats * sizeof(long long));
    std::memcpy(hoffs + 2 * nmats, ooff.data(), nmats * sizeof(long long));
    cudaError_t e;
    // the three offset tables are contiguous in the workspace (o_aoff, o_nmat, o_ooff)
    long long* daoff = reinterpret_cast<long long*>(base + L.o_aoff);
    long long* dnmat = reinterpret_cast<long long*>(base + L.o_nmat);
    long long* dooff = reinterpret_cast<long long*>(base + L.o_ooff);
    double* dsub = reinterpret_cast<double*>(base + L.sub);
    if ((e = cudaMemcpyAsync(daoff, hoffs, nmats * sizeof(long long), cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dnmat, hoffs + nmats, nmats * sizeof(long long), cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(dooff, hoffs + 2 * nmats, nmats * sizeof(long long), cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess)
        return cuda_fail(e, "batched: upload offsets");
    if (L.nsub > 0) {
        if ((e = launch_batch_subdiag(daoff, dnmat, dooff, static_cast<int>(nmats), maxn, A_pool, dsub, stream)) !=
            cudaSuccess)
            return cuda_fail(e, "batched: gather sub-diagonals");
        if ((e = cudaMemcpyAsync(hsub, dsub, L.nsub * sizeof(double), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
            return cuda_fail(e, "batched: read sub-diagonals");
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "batched: synchronize before planning");
    sub.assign(L.nsub + 1, 0);
    {
        size_t k = 0, so = 0;
        for (int q = 0; q < count; q++)
            for (int mu = 0; mu < d[q]; mu++, k++) {
                const long long m = n_packed[k];
                for (long long i = 0; i + 1 < m; i++) sub[so + i] = hsub[so + i] != 0.0 ? 1 : 0;
                for (long long i = 0; i + 2 < m; i++)
                    if (sub[so + i] && sub[so + i + 1]) {
                        if (per_status)
                            for (int r = 0; r < count; r++) per_status[r] = r == q ? -6 : 0;
                        return -6;  // not quasi-triangular
                    }
                so += static_cast<size_t>(m - 1);
            }
    }

    return 0;
}


// ------------------------------------------------ batched mixed-precision refinement
//
// All equations of one order d (the pooled elementwise kernels need one block
// size).  FP32 side: the batch plan with 4-byte entries (block tensors pooled,
// FP32 coefficient tiles, the persistent FP32 solve).  FP64 side, after it in
// the workspace: pooled B, X, R block tensors, FP64 coefficient tiles, the
// Horner intermediates of the generalized residual, block and equation norms.
struct RefExtra {
    size_t Bt = 0, Xt = 0, Rt = 0, set[2][2] = {}, part = 0, xpart = 0, nrm = 0, nA = 0;
    size_t tab = 0, tab_bytes = 0;  // geo64, geoX, args[2][4][count], ajobs, tile_eq, tile_off, norm tables
    size_t o_geo64 = 0, o_geoX = 0, o_args = 0, o_ajobs = 0, o_teq = 0, o_toff = 0, o_noff = 0, o_nn = 0, o_nup = 0;
    size_t coef = 0, coef_bytes = 0;  // FP64 coefficient tiles
    size_t cfh = 0, cfl = 0;          // their float-pair split (the first step's DF64 residual)
    size_t total = 0;
};

RefExtra make_ref_extra(size_t start, int count, int d, bool gen, long long tiles, long long ctiles, int nmats) {
    RefExtra E;
    const int te = tile_extent(d);
    const size_t td = static_cast<size_t>(ipow(te, d)), tc = static_cast<size_t>(te) * te;
    const bool g = gen && d >= 2;
    size_t o = al256(start);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = al256(o + bytes);
        return at;
    };
    E.Bt = take(tiles * td * 8);
    E.Xt = take(tiles * td * 8);
    E.Rt = take(tiles * td * 8);
    if (g)
        for (int k = 0; k < 2; k++)
            for (int j = 0; j < 2; j++) E.set[k][j] = take(tiles * td * 8);
    E.part = take(tiles * 2 * 8);
    E.xpart = take(tiles * 8);
    E.nrm = take(static_cast<size_t>(count) * 4 * 8);
    E.nA = take(static_cast<size_t>(nmats) * 8);
    E.coef_bytes = static_cast<size_t>(ctiles) * tc * 8 * (g ? 2 : 1) + static_cast<size_t>(count) * d * 2 * 256;
    E.coef = take(E.coef_bytes);
    E.cfh = take(E.coef_bytes / 2);
    E.cfl = take(E.coef_bytes / 2);
    size_t t = 0;
    auto tt = [&](size_t bytes) {
        const size_t at = t;
        t = al256(t + bytes);
        return at;
    };
    E.o_geo64 = tt(count * sizeof(BatchGeom));
    E.o_geoX = tt(count * sizeof(BatchGeom));
    E.o_args = tt(static_cast<size_t>(3) * kMaxD * count * sizeof(ApplyArgs));
    E.o_ajobs = tt(tiles * sizeof(int2));
    E.o_teq = tt(tiles * sizeof(int));
    E.o_toff = tt((count + 1) * sizeof(long long));
    E.o_noff = tt(static_cast<size_t>(nmats) * sizeof(long long));
    E.o_nn = tt(static_cast<size_t>(nmats) * sizeof(long long));
    E.o_nup = tt(static_cast<size_t>(nmats) * sizeof(int));
    E.tab_bytes = t;
    E.tab = take(t);
    E.total = o;
    return E;
}

bool uniform_order(int count, const int* d) {
    for (int e = 1; e < count; e++)
        if (d[e] != d[0]) return false;
    return true;
}

// Fixed tile shape of the options (opts->nmin > 0 or opts->leaf), else -1.
// Every equation of a batch takes the same per-mode bounds (each clipped to
// its own order's tile extent).
int fixed_shape_of(const tsylv_opts& o) {
    bool per_mode = false;
    for (int mu = 0; mu < kMaxD; mu++) per_mode |= o.leaf[mu] > 0;
    if (!per_mode) return o.nmin > 0 ? kShapeFixed + o.nmin : -1;
    const int dflt = o.nmin > 0 ? o.nmin : 63;
    int code = 0;
    for (int mu = 0; mu < kMaxD; mu++) code |= (o.leaf[mu] > 0 ? o.leaf[mu] : dflt) << (6 * mu);
    return kShapeFixed + code;
}

// The FP64 batch tunes the tile shape with its launch (-1 marks "any
// candidate" for the workspace bounds) unless the options fix it.
int fp64_shape(const tsylv_opts& o) { return fixed_shape_of(o); }

// The FP32-refined batch runs one fixed tile shape: the default, or the options'.
int refined_shape(const tsylv_opts& o) {
    const int f = fixed_shape_of(o);
    return f >= 0 ? f : 0;
}

size_t refined_workspace_bytes(int count, const int* d, const int64_t* n_packed, bool gen, int shape) {
    const Bounds b = batch_bounds(count, d, n_packed, gen, 4, shape);
    const BatchLayout L = make_batch_layout(count, d, n_packed, gen, 4, b.jobs, b.cjobs, b.pints, b.data);
    int nm = 0;
    for (int e = 0; e < count; e++) nm += d[e] * (gen ? 2 : 1);
    return make_ref_extra(L.total, count, d[0], gen, b.jobs, b.cjobs, nm).total;
}

thread_local Pinned t_pin_nrm;

int solver_batched_refined(int count, const int* d, const int64_t* n_packed, const int64_t* off_A,
                           const int64_t* off_X, const double* A_pool, const double* C_pool, const double* B_pool,
                           double* X_pool, char* base, size_t work_bytes, const tsylv_opts& o,
                           const std::vector<uint8_t>& sub, int* herr, int* per_status, tsylv_info* info,
                           cudaStream_t stream) {
    const bool gen = C_pool != nullptr;
    const int dd = d[0];
    const bool g = gen && dd >= 2;
    const int te = tile_extent(dd), td = ipow(te, dd), tc = te * te;
    const int shape = refined_shape(o);
    const Bounds bd = batch_bounds(count, d, n_packed, gen, 4, shape);
    const BatchLayout L = make_batch_layout(count, d, n_packed, gen, 4, bd.jobs, bd.cjobs, bd.pints, bd.data);
    const int nmA = count * dd, nm = nmA * (gen ? 2 : 1);
    std::shared_ptr<BatchPlan> plan =
        get_batch_plan(count, d, n_packed, gen, 4, sub, o.partition == 1 ? 1 : 0, shape);
    if (!plan) return cuda_fail_msg("batched: plan");
    if (plan->data_bytes > bd.data) return cuda_fail_msg("batched: workspace bound");
    const long long T = plan->tile_off[count];
    long long ctiles = 0;
    for (const EqPlan& q : plan->eq)
        for (int mu = 0; mu < q.d; mu++) ctiles += static_cast<long long>(q.nb[mu]) * (q.nb[mu] + 1) / 2;
    const RefExtra E = make_ref_extra(L.total, count, dd, gen, bd.jobs, bd.cjobs, nm);
    if (E.total > work_bytes) return -11;
    if (int st = prepare_batched_once()) return st;

    // ---- host tables: the FP32 solve's (as a plain batched solve), then the FP64 side's
    std::vector<unsigned char> tabv;
    const int policy = plan->tuned_policy >= 0 ? plan->tuned_policy : 0;
    fill_table(*plan, L, base, policy, tabv, off_A, off_X);
    std::vector<unsigned char> xt(E.tab_bytes, 0);
    BatchGeom* g64 = reinterpret_cast<BatchGeom*>(xt.data() + E.o_geo64);
    BatchGeom* gX = reinterpret_cast<BatchGeom*>(xt.data() + E.o_geoX);
    // [mode 0 full FP64, 1 FP32 update, 2 first step in DF64 on the FP32 correction][level][eq]
    ApplyArgs* args = reinterpret_cast<ApplyArgs*>(xt.data() + E.o_args);
    int2* ajobs = reinterpret_cast<int2*>(xt.data() + E.o_ajobs);
    int* teq = reinterpret_cast<int*>(xt.data() + E.o_teq);
    long long* toff = reinterpret_cast<long long*>(xt.data() + E.o_toff);
    long long* noff = reinterpret_cast<long long*>(xt.data() + E.o_noff);
    long long* nn = reinterpret_cast<long long*>(xt.data() + E.o_nn);
    int* nup = reinterpret_cast<int*>(xt.data() + E.o_nup);
    const BatchGeom* g32 = reinterpret_cast<const BatchGeom*>(tabv.data() + L.o_geom);
    const WaveArgs* w32 = reinterpret_cast<const WaveArgs*>(tabv.data() + L.o_wave);
    char* dt = base + E.tab;
    double* Bt = reinterpret_cast<double*>(base + E.Bt);
    double* Xt = reinterpret_cast<double*>(base + E.Xt);
    double* Rt = reinterpret_cast<double*>(base + E.Rt);
    double* part = reinterpret_cast<double*>(base + E.part);
    double* xpart = reinterpret_cast<double*>(base + E.xpart);
    double* nrm = reinterpret_cast<double*>(base + E.nrm);
    double* nA = reinterpret_cast<double*>(base + E.nA);
    int* errs = reinterpret_cast<int*>(base + L.ctl) + 8 + count;
    size_t coff = E.coef;
    size_t k = 0;
    for (int e = 0; e < count; e++) {
        const EqPlan& q = plan->eq[e];
        const long long t0 = plan->tile_off[e];
        toff[e] = t0;
        for (long long t = 0; t < q.ntiles; t++) {
            ajobs[t0 + t] = make_int2(e, static_cast<int>(t));
            teq[t0 + t] = e;
        }
        BatchGeom a = g32[e];
        a.X = Bt + t0 * td;
        for (int mu = 0; mu < dd; mu++, k++) {
            const size_t bytes = static_cast<size_t>(q.nb[mu]) * (q.nb[mu] + 1) / 2 * tc * 8;
            a.At[mu] = base + coff;
            coff = al256(coff + bytes);
            a.Ct[mu] = nullptr;
            if (g) {
                a.Ct[mu] = base + coff;
                coff = al256(coff + bytes);
            }
            noff[e * dd + mu] = off_A[k];
            nn[e * dd + mu] = q.n[mu];
            nup[e * dd + mu] = 0;
            if (gen) {
                noff[nmA + e * dd + mu] = off_A[k];
                nn[nmA + e * dd + mu] = q.n[mu];
                nup[nmA + e * dd + mu] = 1;
            }
        }
        g64[e] = a;
        BatchGeom x = a;
        x.X = Xt + t0 * td;
        gX[e] = x;
        // residual applies: [0] full FP64 R = B - A(X), [1] FP32 update R -= s A(D),
        // [2] the first step (X = s D exactly): R = B - s A(D) in DF64 on the
        // FP32 correction D, the coefficients as float pairs, the d-term
        // form's intermediates as float-pair planes of the FP64 sets
        auto cf = [&](const void* p64, size_t region) -> const void* {
            return base + region + static_cast<size_t>(static_cast<const char*>(p64) - (base + E.coef)) / 2;
        };
        for (int mode = 0; mode < 3; mode++) {
            const int levels = g ? dd : 1;
            int cur = 0;
            for (int lv = 0; lv < levels; lv++) {
                ApplyArgs r{};
                for (int mu = 0; mu < dd; mu++) {
                    r.nb[mu] = q.nb[mu];
                    r.tstride[mu] = q.tstride[mu];
                    if (mode == 2) {
                        r.A[mu] = cf(a.At[mu], E.cfh);
                        r.Al[mu] = cf(a.At[mu], E.cfl);
                        r.C[mu] = g ? cf(a.Ct[mu], E.cfh) : nullptr;
                        r.Cl[mu] = g ? cf(a.Ct[mu], E.cfl) : nullptr;
                    } else {
                        r.A[mu] = mode == 0 ? a.At[mu] : w32[e].At[mu];
                        r.C[mu] = g ? (mode == 0 ? a.Ct[mu] : w32[e].Ct[mu]) : nullptr;
                    }
                }
                r.ntiles = q.ntiles;
                r.B = mode == 1 ? Rt + t0 * td : Bt + t0 * td;
                r.R = Rt + t0 * td;
                r.scale = mode == 0 ? nullptr : nrm + 4 * e;
                r.part = part + 2 * t0;
                r.err = errs + e;
                r.timeout_ns = t_timeout_ns;
                const void* xs = mode == 0 ? static_cast<const void*>(Xt + t0 * td) : w32[e].X;
                auto setp = [&](int kk, int j) -> void* {
                    return base + E.set[kk][j] + static_cast<size_t>(t0) * td * 8;
                };
                // float-pair planes of set kk, j: the high words, then the low words
                auto seth = [&](int kk, int j) -> void* {
                    return base + E.set[kk][j] + static_cast<size_t>(t0) * td * 4;
                };
                auto setl = [&](int kk, int j) -> void* {
                    return base + E.set[kk][j] + static_cast<size_t>(T) * td * 4 + static_cast<size_t>(t0) * td * 4;
                };
                if (!g) {
                    r.kind = kApplyLaplace;
                    r.s1 = xs;
                } else if (lv == 0) {
                    r.kind = kApplyFirst;
                    r.mode = dd - 1;
                    r.s1 = xs;
                    if (mode == 2) {
                        r.o1 = seth(0, 0);
                        r.o1l = setl(0, 0);
                        r.o2 = seth(0, 1);
                        r.o2l = setl(0, 1);
                    } else {
                        r.o1 = setp(0, 0);
                        r.o2 = setp(0, 1);
                    }
                    cur = 0;
                } else {
                    const int l = dd - 1 - lv;  // mode of this level
                    r.kind = l == 0 ? kApplyFinal : kApplyMiddle;
                    r.mode = l;
                    if (mode == 2) {
                        r.s1 = seth(cur, 0);
                        r.s1l = setl(cur, 0);
                        r.s2 = seth(cur, 1);
                        r.s2l = setl(cur, 1);
                        r.o1 = seth(1 - cur, 0);
                        r.o1l = setl(1 - cur, 0);
                        r.o2 = seth(1 - cur, 1);
                        r.o2l = setl(1 - cur, 1);
                    } else {
                        r.s1 = setp(cur, 0);
                        r.s2 = setp(cur, 1);
                        r.o1 = setp(1 - cur, 0);
                        r.o2 = setp(1 - cur, 1);
                    }
                    cur = 1 - cur;
                }
                args[(static_cast<size_t>(mode) * kMaxD + lv) * count + e] = r;
            }
        }
    }
    toff[count] = T;
    const size_t tab_all = L.tab_bytes + E.tab_bytes;
    if (!t_pin_tab.reserve(tab_all)) return cuda_fail_msg("batched: pinned host allocation");
    std::memcpy(t_pin_tab.ptr, tabv.data(), L.tab_bytes);
    std::memcpy(t_pin_tab.ptr + L.tab_bytes, xt.data(), E.tab_bytes);
    if (!t_pin_nrm.reserve(static_cast<size_t>(count) * 4 * 8 + static_cast<size_t>(nm) * 8))
        return cuda_fail_msg("batched: pinned host allocation");
    double* hn = reinterpret_cast<double*>(t_pin_nrm.ptr);
    double* hA = hn + 4 * count;

    int per_sm = o.split > 0 ? o.split : occupancy_cached(dd, gen, 4);
    per_sm = std::max(1, std::min(per_sm, occupancy_cached(dd, gen, 4)));
    int grid = per_sm * sm_count();
    if (grid > T) grid = static_cast<int>(T);
    if (grid < 1) grid = 1;
    char* tab32 = base + L.tab;
    const BatchGeom* dgeo32 = reinterpret_cast<const BatchGeom*>(tab32 + L.o_geom);
    const BatchJob* djobs = reinterpret_cast<const BatchJob*>(tab32 + L.o_jobs);
    const BatchCoefJob* dcjobs = reinterpret_cast<const BatchCoefJob*>(tab32 + L.o_cjobs);
    const BatchGeom* dgeo64 = reinterpret_cast<const BatchGeom*>(dt + E.o_geo64);
    const BatchGeom* dgeoX = reinterpret_cast<const BatchGeom*>(dt + E.o_geoX);
    const ApplyArgs* dargs = reinterpret_cast<const ApplyArgs*>(dt + E.o_args);
    const int2* dajobs = reinterpret_cast<const int2*>(dt + E.o_ajobs);
    const int* dteq = reinterpret_cast<const int*>(dt + E.o_teq);
    const long long* dtoff = reinterpret_cast<const long long*>(dt + E.o_toff);
    const long long* dnoff = reinterpret_cast<const long long*>(dt + E.o_noff);
    const long long* dnn = reinterpret_cast<const long long*>(dt + E.o_nn);
    const int* dnup = reinterpret_cast<const int*>(dt + E.o_nup);
    int* ctl = reinterpret_cast<int*>(base + L.ctl);
    const int njobs = static_cast<int>(plan->jobs[0].size());
    const int ncj = static_cast<int>(plan->cjobs.size());
    long long nmax = 1;
    for (int q = 0; q < nm; q++) nmax = std::max(nmax, nn[q]);
    float* X32 = static_cast<float*>(w32[0].X);  // the pooled FP32 block tensors start with equation 0

#define TRYB(x)                               \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)
    auto setup = [&](cudaStream_t s) -> cudaError_t {
        TRYB(cudaMemsetAsync(ctl, 0, (8 + 2 * static_cast<size_t>(count)) * sizeof(int), s));
        TRYB(cudaMemcpyAsync(tab32, t_pin_tab.ptr, L.tab_bytes, cudaMemcpyHostToDevice, s));
        TRYB(cudaMemcpyAsync(dt, t_pin_tab.ptr + L.tab_bytes, E.tab_bytes, cudaMemcpyHostToDevice, s));
        TRYB(launch_batch_pack<float>(dgeo32, djobs, 0, dcjobs, ncj, nullptr, A_pool, C_pool, s));
        TRYB(launch_batch_pack<double>(dgeo64, djobs, njobs, dcjobs, ncj, B_pool, A_pool, C_pool, s));
        TRYB(launch_split(reinterpret_cast<const double*>(base + E.coef), reinterpret_cast<float*>(base + E.cfh),
                          reinterpret_cast<float*>(base + E.cfl), static_cast<long long>(E.coef_bytes / 8), s));
        TRYB(cudaMemsetAsync(Xt, 0, static_cast<size_t>(T) * td * 8, s));
        TRYB(cudaMemcpyAsync(Rt, Bt, static_cast<size_t>(T) * td * 8, cudaMemcpyDeviceToDevice, s));
        TRYB(launch_tile_stats(Rt, part, T, td, s));
        TRYB(launch_breduce(part, nullptr, dtoff, count, nrm, s));
        TRYB(launch_bnorm2(A_pool, dnoff, dnn, dnup, nmA, nmax, nA, s));
        if (gen) TRYB(launch_bnorm2(C_pool, dnoff + nmA, dnn + nmA, dnup + nmA, nmA, nmax, nA + nmA, s));
        TRYB(cudaMemcpyAsync(hn, nrm, static_cast<size_t>(count) * 4 * 8, cudaMemcpyDeviceToHost, s));
        return cudaMemcpyAsync(hA, nA, static_cast<size_t>(nm) * 8, cudaMemcpyDeviceToHost, s);
    };
    auto iterate = [&](bool update, bool first, cudaStream_t s) -> cudaError_t {
        TRYB(launch_bscale(Rt, X32, dteq, nrm, T * td, td, s));
        TRYB(cudaMemsetAsync(ctl, 0, 8 * sizeof(int) + static_cast<size_t>(count) * sizeof(int), s));
        TRYB(cudaMemsetAsync(base + L.flags, 0, static_cast<size_t>(T) * sizeof(int), s));
        BatchArgs ba{};
        ba.eqs = reinterpret_cast<const WaveArgs*>(tab32 + L.o_wave);
        ba.jobs = djobs;
        ba.njobs = njobs;
        ba.head = ctl;
        ba.abort = ctl + 4;
        ba.done = ctl + 8;
        ba.timeout_ns = t_timeout_ns;
        TRYB(launch_batched<float>(dd, gen, ba, grid, s));
        TRYB(launch_bupdate(Xt, X32, dteq, nrm, xpart, T, td, s));
        const int levels = g ? dd : 1;
        const int mode = update ? 1 : first ? 2 : 0;
        for (int lv = 0; lv < levels; lv++) {
            const int am = update ? kModeF32 : !first ? kModeF64 : lv == 0 ? kModeDFh : kModeDF;
            TRYB(launch_apply_batched(dd, am, dargs + (static_cast<size_t>(mode) * kMaxD + lv) * count, dajobs,
                                      static_cast<int>(T), s));
        }
        TRYB(launch_breduce(part, xpart, dtoff, count, nrm, s));
        return cudaMemcpyAsync(hn, nrm, static_cast<size_t>(count) * 4 * 8, cudaMemcpyDeviceToHost, s);
    };
    auto finish = [&](cudaStream_t s) -> cudaError_t {
        TRYB(launch_batch_unpack<double>(dgeoX, djobs, njobs, X_pool, s));
        return cudaMemcpyAsync(herr, errs, sizeof(int) * count, cudaMemcpyDeviceToHost, s);
    };
#undef TRYB

    std::vector<const void*> kb = {base, A_pool, C_pool, B_pool, X_pool, t_pin_tab.ptr, t_pin_nrm.ptr, herr,
                                   reinterpret_cast<const void*>(static_cast<uintptr_t>(per_sm)),
                                   reinterpret_cast<const void*>(static_cast<uintptr_t>(t_timeout_ns))};
    auto key = [&](int tag) {
        std::vector<const void*> kk = kb;
        kk.push_back(reinterpret_cast<const void*>(static_cast<uintptr_t>(1000 + tag)));
        return kk;
    };
    const bool ug = o.use_graph != 0;
    if (int st = run_graph(*plan, key(0), ug, stream, setup, "batched refinement: set-up")) return st;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "batched refinement: synchronize");
    std::vector<double> normA(count, 0.0), rho(count, -1.0);
    for (int q = 0; q < count; q++) {
        double s = 0;
        for (int mu = 0; mu < dd; mu++) {
            double t = hA[q * dd + mu];
            if (gen)
                for (int eta = 0; eta < dd; eta++)
                    if (eta != mu) t *= hA[nmA + q * dd + eta];
            s += t;
        }
        normA[q] = s;
    }
    std::vector<char> zero(count, 0);
    for (int q = 0; q < count; q++) zero[q] = !(hn[4 * q + 1] > 0);
    int iters = 0, stall = 0;
    double prev = HUGE_VAL, worst = 0;
    bool update = false;
    for (int it = 0; it < std::max(1, o.max_refine); it++) {
        if (o.resid_update == 0 && it > 0 && prev <= 1e-5) update = true;
        const bool first = it == 0;
        if (int st = run_graph(*plan, key(update ? 2 : first ? 4 : 1), ug, stream,
                               [&](cudaStream_t s) { return iterate(update, first, s); }, "batched refinement: step"))
            return st;
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "batched refinement: synchronize");
        iters = it + 1;
        worst = 0;
        bool bad = false;
        for (int q = 0; q < count; q++) {
            const double xn = std::sqrt(hn[4 * q + 2]);
            rho[q] = zero[q] ? 0.0 : (xn > 0 && normA[q] > 0 ? std::sqrt(hn[4 * q]) / (normA[q] * xn) : 0.0);
            if (!std::isfinite(rho[q])) bad = true;
            worst = std::max(worst, rho[q]);
        }
        if (bad || worst <= o.tol) break;
        if (worst > 0.5 * prev) {
            if (++stall >= 2) break;
        } else {
            stall = 0;
        }
        prev = worst;
    }
    if (int st = run_graph(*plan, key(3), ug, stream, finish, "batched refinement: unpack")) return st;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "batched refinement: synchronize");
    int status = TSYLV_OK;
    for (int q = 0; q < count; q++) {
        int s = map_status(herr[q]);
        if (s == TSYLV_OK && !std::isfinite(rho[q])) s = TSYLV_ENONFINITE;
        if (s == TSYLV_OK && !(rho[q] <= o.tol)) s = TSYLV_ENOCONV;
        if (per_status) per_status[q] = s;
        if (status == TSYLV_OK && s != TSYLV_OK) status = s;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        int waves = 0;
        for (const EqPlan& q : plan->eq) waves = std::max(waves, q.nwaves);
        info->iterations = iters;
        info->waves = waves;
        info->launches = 6 + (gen ? 2 : 1) + iters * (4 + (g ? dd : 1)) + 1;
        info->tiles = static_cast<int>(T);
        info->resid = worst;
        info->norm_A = -1;
        info->flops = plan->flops * iters;
        info->batch_order = policy;
        info->batch_ctas_per_sm = per_sm;
        const int dmax = plan->dlist.back();
        for (int mu = 0; mu < dmax; mu++) info->leaf[mu] = shape_cut(dmax, mu, shape);
    }
    (void)ctiles;
    return status;
}
}  // namespace

size_t solver_batched_workspace_bytes(int count, const int* d, const int64_t* n_packed, bool gen,
                                      const tsylv_opts& o) {
    if (!shapes_ok(count, d, n_packed)) return 0;
    if (o.precision == TSYLV_FP32_REFINED)
        return uniform_order(count, d) ? refined_workspace_bytes(count, d, n_packed, gen, refined_shape(o)) : 0;
    if (o.precision != TSYLV_FP64 && o.precision != TSYLV_DF64) return 0;
    const Bounds b = batch_bounds(count, d, n_packed, gen, 8, fp64_shape(o));
    const BatchLayout L = make_batch_layout(count, d, n_packed, gen, 8, b.jobs, b.cjobs, b.pints, b.data);
    return L.total;
}

int solver_batched(int count, const int* d, const int64_t* n_packed, const int64_t* off_A, const int64_t* off_X,
                   const double* A_pool, const double* C_pool, const double* B_pool, double* X_pool, void* work,
                   size_t work_bytes, const tsylv_opts* opts, int* per_status, tsylv_info* info,
                   cudaStream_t stream) {
    tsylv_opts o;
    if (opts) o = *opts; else tsylv_opts_default(&o);
    if (count < 1) return -1;
    if (!d) return -2;
    if (!n_packed || !shapes_ok(count, d, n_packed)) return -3;
    if (!off_A) return -4;
    if (!off_X) return -5;
    if (!A_pool) return -6;
    const bool gen = C_pool != nullptr;
    if (!B_pool) return -8;
    if (!X_pool) return -9;
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255)) return -10;
    if (o.precision != TSYLV_FP64 && o.precision != TSYLV_FP32_REFINED && o.precision != TSYLV_DF64)
        return TSYLV_EUNSUPPORTED;
    const bool refined = o.precision == TSYLV_FP32_REFINED;
    const bool df64 = o.precision == TSYLV_DF64;
    if (df64)  // the double-float kernels are built for d <= 4
        for (int e = 0; e < count; e++)
            if (d[e] > 4) return TSYLV_EUNSUPPORTED;
    if (refined && !uniform_order(count, d)) return TSYLV_EUNSUPPORTED;
    if (gen)  // the generalized form is built for d <= 4
        for (int e = 0; e < count; e++)
            if (d[e] > 4) return TSYLV_EUNSUPPORTED;
    const size_t need = solver_batched_workspace_bytes(count, d, n_packed, gen, o);
    if (!need || work_bytes < need) return -11;
    if (o.split < 0 || o.partition < 0 || o.partition > 1 || o.wait_ms < 1 || o.wait_ms > 600000 || o.nmin < -1 ||
        o.fp64_update < 0 || o.fp64_update > 2)
        return -12;
    if (o.fp64_update == 2) return TSYLV_EUNSUPPORTED;  // the batch runs FMA block updates
    for (int mu = 0; mu < kMaxD; mu++)
        if (o.leaf[mu] < 0) return -12;
    for (int e = 0; e < count; e++) {
        if (o.nmin == 1 || o.nmin > tile_extent(d[e])) return TSYLV_EUNSUPPORTED;
        for (int mu = 0; mu < kMaxD; mu++)
            if (o.leaf[mu] == 1 || (mu < d[e] && o.leaf[mu] > tile_extent(d[e]))) return TSYLV_EUNSUPPORTED;
    }
    t_timeout_ns = static_cast<long long>(o.wait_ms) * 1000000LL;
    size_t nmats = 0;
    for (int e = 0; e < count; e++) nmats += static_cast<size_t>(d[e]);
    for (size_t k = 0; k < nmats; k++)
        if (off_A[k] < 0) return -4;
    for (int e = 0; e < count; e++)
        if (off_X[e] < 0) return -5;
    (void)cudaGetLastError();
    char* base = static_cast<char*>(work);
    const int elem = refined ? 4 : 8;
    const Bounds bd = batch_bounds(count, d, n_packed, gen, elem, refined ? refined_shape(o) : fp64_shape(o));
    BatchLayout L = make_batch_layout(count, d, n_packed, gen, elem, bd.jobs, bd.cjobs, bd.pints, bd.data);

    std::vector<uint8_t> sub;
    int* herr = nullptr;
    if (int st = batch_structure(count, d, n_packed, off_A, A_pool, base, L, per_status, stream, sub, herr)) return st;
    if (refined)
        return solver_batched_refined(count, d, n_packed, off_A, off_X, A_pool, C_pool, B_pool, X_pool, base,
                                      work_bytes, o, sub, herr, per_status, info, stream);
    cudaError_t e;

    // ---- plan (cached per shapes and structure), tables, launch
    const int fixed_shape = fixed_shape_of(o);
    const int part_rule = o.partition == 1 ? 1 : 0;
    std::shared_ptr<BatchPlan> plan0 =
        get_batch_plan(count, d, n_packed, gen, 8, sub, part_rule, fixed_shape >= 0 ? fixed_shape : 0, df64 ? 1 : 0);
    if (!plan0) return cuda_fail_msg("batched: plan");
    if (plan0->data_bytes > bd.data) return cuda_fail_msg("batched: workspace bound");
    if (int st = prepare_batched_once()) return st;
    BatchCall c;
    c.df64 = df64;
    c.plan = plan0.get();
    c.L = L;
    c.base = base;
    c.A = A_pool;
    c.C = C_pool;
    c.B = B_pool;
    c.X = X_pool;
    c.herr = herr;
    if (!t_pin_tab.reserve(L.tab_bytes)) return cuda_fail_msg("batched: pinned host allocation");
    std::vector<unsigned char> tabv;

    auto set_grid = [&](int per_sm) {
        for (int dd : plan0->dlist) {
            const int occ = occupancy_cached(dd, gen, 8, df64);
            c.grid_per_sm[dd] = std::max(1, std::min(per_sm, occ));
        }
    };

    // autotuner: tile shape (the recursion cutoff of every mode) x queue order
    // x resident CTAs per SM, timed on this batch once (the persistent launches
    // with CUDA events; the timing runs leave X_pool untouched)
    int shape = fixed_shape >= 0 ? fixed_shape : plan0->tuned_shape;
    int policy = plan0->tuned_policy, per_sm = plan0->tuned_grid;
    std::shared_ptr<BatchPlan> plan = plan0;
    if (o.split > 0) {
        shape = fixed_shape >= 0 ? fixed_shape : 0;
        policy = policy >= 0 ? policy : 0;
        per_sm = o.split;
    } else if (policy < 0) {
        int occ = 1;
        for (int dd : plan0->dlist) occ = std::max(occ, occupancy_cached(dd, gen, 8, df64));
        std::vector<int> grids = {occ};
        if (occ >= 2) grids.push_back((occ + 1) / 2);
        if (occ >= 3) grids.push_back(1);
        std::vector<int> shapes;
        if (fixed_shape >= 0) {
            shapes.push_back(fixed_shape);
        } else {
            const bool only_d1 = plan0->dlist.size() == 1 && plan0->dlist[0] == 1;
            for (int sc = 0; sc < kShapes; sc++)
                if (!(only_d1 && sc >= 4)) shapes.push_back(sc);  // 4 coincides with 3 for one mode
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return cuda_fail_msg("batched: autotuner events");
        }
        float best = 1e30f;
        int bs = shapes[0], bp = 0, bg = occ;
        for (int sc : shapes) {
            std::shared_ptr<BatchPlan> ps =
                sc == (fixed_shape >= 0 ? fixed_shape : 0) ? plan0 : get_batch_plan(count, d, n_packed, gen, 8, sub,
                                                                                     part_rule, sc, df64 ? 1 : 0);
            if (!ps || ps->data_bytes > bd.data) continue;
            c.plan = ps.get();
            c.L = plan_layout(*ps, d, n_packed, 8);
            if (c.L.total > L.total) continue;
            for (int pol = 0; pol < kPolicies; pol++) {
                fill_table(*ps, c.L, base, pol, tabv, off_A, off_X);
                std::memcpy(t_pin_tab.ptr, tabv.data(), tabv.size());
                c.htab = t_pin_tab.ptr;
                for (int gsz : grids) {
                    set_grid(gsz);
                    c.ev0 = e0;
                    c.ev1 = e1;
                    c.unpack = false;  // the timing runs leave X_pool (which may be B_pool) untouched
                    float ms = 1e30f;
                    for (int rep = 0; rep < 3; rep++) {  // first run warms caches and code; best of two after it
                        if ((e = enqueue_batch(c, stream)) != cudaSuccess) {
                            cudaEventDestroy(e0);
                            cudaEventDestroy(e1);
                            return cuda_fail(e, "batched: autotuner launch");
                        }
                        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) {
                            cudaEventDestroy(e0);
                            cudaEventDestroy(e1);
                            return cuda_fail(e, "batched: autotuner synchronize");
                        }
                        float t = 1e30f;
                        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) t = 1e30f;
                        if (rep > 0 && t < ms) ms = t;
                    }
                    int bad = 0;
                    for (int q = 0; q < count; q++) bad |= herr[q];
                    if (bad & kErrTimeout) ms = 1e30f;
                    if (ms < best) {
                        best = ms;
                        bs = sc;
                        bp = pol;
                        bg = gsz;
                    }
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c.ev0 = c.ev1 = nullptr;
        c.unpack = true;
        plan0->tuned_shape = shape = bs;
        plan0->tuned_policy = policy = bp;
        plan0->tuned_grid = per_sm = bg;
    }
    if (shape != (fixed_shape >= 0 ? fixed_shape : 0)) {
        plan = get_batch_plan(count, d, n_packed, gen, 8, sub, part_rule, shape, df64 ? 1 : 0);
        if (!plan) return cuda_fail_msg("batched: plan");
        if (plan->data_bytes > bd.data) return cuda_fail_msg("batched: workspace bound");
    }
    c.plan = plan.get();
    c.L = plan_layout(*plan, d, n_packed, 8);
    if (c.L.total > L.total) return cuda_fail_msg("batched: workspace bound");
    set_grid(per_sm);
    fill_table(*plan, c.L, base, policy, tabv, off_A, off_X);
    std::memcpy(t_pin_tab.ptr, tabv.data(), tabv.size());
    c.htab = t_pin_tab.ptr;

    const int launches = 3 + static_cast<int>(plan->dlist.size());
    if (o.use_graph) {
        std::vector<const void*> key = {base, A_pool, C_pool, B_pool, X_pool, t_pin_tab.ptr, herr,
                                        reinterpret_cast<const void*>(static_cast<uintptr_t>(policy * 64 + per_sm)),
                                        reinterpret_cast<const void*>(static_cast<uintptr_t>(t_timeout_ns))};
        cudaGraphExec_t exec = nullptr;
        for (auto& g : plan->graphs)
            if (g.key == key) exec = g.exec;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            cudaStream_t cs = capture_stream();
            if (!cs) return cuda_fail_msg("batched: capture stream");
            if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "batched: begin capture");
            const cudaError_t ee = enqueue_batch(c, cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(ee, "batched: capture");
            }
            if (e != cudaSuccess) return cuda_fail(e, "batched: end capture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "batched: instantiate");
            if (plan->graphs.size() >= 8) {
                cudaGraphExecDestroy(plan->graphs.front().exec);
                plan->graphs.erase(plan->graphs.begin());
            }
            plan->graphs.push_back({key, exec});
        }
        if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return cuda_fail(e, "batched: graph launch");
    } else {
        if ((e = enqueue_batch(c, stream)) != cudaSuccess) return cuda_fail(e, "batched: launch");
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "batched: synchronize");
    int status = TSYLV_OK;
    for (int q = 0; q < count; q++) {
        const int s = map_status(herr[q]);
        if (per_status) per_status[q] = s;
        if (status == TSYLV_OK && s != TSYLV_OK) status = s;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        int waves = 0;
        long long tiles = 0;
        for (const EqPlan& q : plan->eq) {
            waves = std::max(waves, q.nwaves);
            tiles += q.ntiles;
        }
        info->waves = waves;
        info->launches = launches;
        info->tiles = static_cast<int>(tiles);
        info->resid = -1;
        info->norm_A = -1;
        info->flops = plan->flops;
        info->batch_order = policy;
        info->batch_ctas_per_sm = per_sm;
        const int dmax = plan->dlist.back();
        for (int mu = 0; mu < dmax; mu++) info->leaf[mu] = shape_cut(dmax, mu, shape);
    }
    return status;
}

}  // namespace tsylv
