// Split tree (Alg. 2), block grid, wavefronts and workspace layout.
#include "plan.h"

#include <algorithm>
#include <cstring>
#include <functional>
#include <numeric>

namespace tsylv {

namespace {

void split_rec(const std::vector<uint8_t>& sub, int lo, int m, int te, std::vector<int>& starts) {
    if (m <= te) {
        starts.push_back(lo);
        return;
    }
    int k = m / 2;
    if (sub[lo + k - 1]) k += 1;  // A(k+1, k) != 0: moving the split keeps the 2x2 block whole
    split_rec(sub, lo, k, te, starts);
    split_rec(sub, lo + k, m - k, te, starts);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Leaf boundaries of one mode.  rule 0 (aligned): blocks of te entries from
// the start, a boundary moved back by one where it would cut a 2x2 block (so
// every block has te or te - 1 entries, the last one possibly fewer: the least
// padding of the te-wide tiles).  rule 1: the split rule of Alg. 2,
// applied recursively (halving, moved by one at a 2x2 block) until every piece
// has at most te entries.  Both partitions keep every 2x2 block whole, so
// they give the same solution up to rounding.
Part make_part(int n, const std::vector<uint8_t>& sub, int te, int rule) {
    Part p;
    p.n = n;
    if (rule == 1) {
        split_rec(sub, 0, n, te, p.start);
    } else {
        int start = 0;
        while (start < n) {
            p.start.push_back(start);
            int end = std::min(start + te, n);
            if (end < n && sub[end - 1]) end -= 1;  // A(end+1, end) != 0 (1-based): keep the 2x2 block whole
            start = end;
        }
    }
    p.nb = static_cast<int>(p.start.size());
    p.size.resize(p.nb);
    p.blk_of.resize(n);
    for (int I = 0; I < p.nb; I++) {
        const int e = I + 1 < p.nb ? p.start[I + 1] : n;
        p.size[I] = e - p.start[I];
        for (int i = p.start[I]; i < e; i++) p.blk_of[i] = I;
    }
    return p;
}

// Largest number of leaves either rule can produce for any admissible structure.
int max_blocks(int n, int te) {
    std::vector<int> memo(static_cast<size_t>(n) + 1, -1);
    std::function<int(int)> f = [&](int m) -> int {
        if (m <= te) return 1;
        if (memo[m] >= 0) return memo[m];
        const int k = m / 2;
        int best = f(k) + f(m - k);
        if (k + 1 < m) best = std::max(best, f(k + 1) + f(m - k - 1));
        memo[m] = best;
        return best;
    };
    // aligned rule: every block but the last has at least te - 1 entries
    const int aligned = te > 1 ? (n - 1) / (te - 1) + 1 : n;
    return std::max(f(n), aligned);
}

int shape_cut(int d, int mu, int shape) {
    const int te = tile_extent(d);
    if (shape >= kShapeFixed) {  // fixed bounds: 6 bits per mode, a zero field takes mode 1's
        const int code = shape - kShapeFixed;
        int c = (code >> (6 * mu)) & 63;
        if (c == 0) c = code & 63;
        return std::max(2, std::min(te, c));
    }
    const int half = std::max(2, te / 2), three = std::max(2, (3 * te) / 4), less = std::max(2, te - 1);
    switch (shape) {
        case 1: return less;
        case 2: return three;
        case 3: return half;
        case 4: return mu == d - 1 ? half : te;
        default: return te;
    }
}

int shape_min_cut(int d, int mu, int shape) {
    if (shape >= 0) return shape_cut(d, mu, shape);
    int c = tile_extent(d);
    for (int s = 0; s < kShapes; s++) c = std::min(c, shape_cut(d, mu, s));
    return c;
}

Plan::~Plan() {
    for (auto& g : graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h_tab) cudaFreeHost(h_tab);
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
}

Layout make_layout(int d, const long long* n, const int* nb, bool gen, int elem, size_t tab_ints, bool tt) {
    Layout L;
    const int te = tile_extent(d);
    const size_t td = static_cast<size_t>(ipow(te, d)), tc = static_cast<size_t>(te) * te;
    size_t ntiles = 1, nsub = 0;
    for (int mu = 0; mu < d; mu++) {
        ntiles *= static_cast<size_t>(nb[mu]);
        nsub += static_cast<size_t>(n[mu] > 0 ? n[mu] - 1 : 0);
    }
    size_t o = 0;
    L.err = o;
    o = align256(o + 64);
    L.sub = o;
    o = align256(o + (nsub + 1) * sizeof(double));
    L.tab = o;
    o = align256(o + tab_ints * sizeof(int));
    L.X = o;
    o = align256(o + ntiles * td * elem);
    if (gen || tt)
        for (int l = 1; l < d; l++) {
            L.P[l] = o;
            o = align256(o + ntiles * td * elem);
            if (tt) continue;
            L.G[l] = o;
            o = align256(o + ntiles * td * elem);
        }
    for (int mu = 0; mu < d; mu++) {
        const size_t ntri = static_cast<size_t>(nb[mu]) * (nb[mu] + 1) / 2;
        L.At[mu] = o;
        o = align256(o + ntri * tc * elem);
        if (gen || (tt && mu == 0)) {
            L.Ct[mu] = o;
            o = align256(o + ntri * tc * elem);
        }
    }
    L.fargs = o;
    o = align256(o + sizeof(WaveArgs));
    L.fctl = o;
    o = align256(o + 64);
    L.flags = o;
    o = align256(o + ntiles * sizeof(int));
    L.total = o;
    return L;
}

namespace {

std::mutex g_mutex;
std::map<std::string, std::shared_ptr<Plan>> g_plans;

void build_waves(Plan& p, int split) {
    const int d = p.d;
    // anti-diagonal index s = sum_mu I_mu; blocks of equal s are independent
    int smax = 0;
    for (int mu = 0; mu < d; mu++) smax += p.nb[mu] - 1;
    std::vector<std::vector<int>> by_s(static_cast<size_t>(smax) + 1);
    std::vector<long long> cost(static_cast<size_t>(p.ntiles));
    for (long long t = 0; t < p.ntiles; t++) {
        int s = 0;
        long long c = 0;
        for (int mu = 0; mu < d; mu++) {
            const int I = static_cast<int>((t / p.tstride[mu]) % p.nb[mu]);
            s += I;
            const int w = p.tt ? (mu == 0 ? 2 : 1) : p.gen && d >= 2 ? ((mu == 0 || mu == d - 1) ? 2 : 3) : 1;
            c += static_cast<long long>(p.nb[mu] - 1 - I) * w;
        }
        by_s[s].push_back(static_cast<int>(t));
        cost[t] = c;
    }
    p.wave_tiles.clear();
    p.wave_off.clear();
    p.wave_cnt.clear();
    p.wave_csize.clear();
    const int cap = split > 0 ? std::min(split, kMaxCluster) : kMaxCluster;
    for (int s = smax; s >= 0; s--) {
        auto& v = by_s[s];
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        long long wmax = 0;
        for (int t : v) wmax = std::max(wmax, cost[t]);
        const long long nt = static_cast<long long>(v.size());
        // split the block updates over a cluster when the wavefront alone
        // cannot fill the GPU twice over, keeping >= 2 jobs' weight per CTA
        long long c = (2LL * 152 + nt - 1) / nt;
        c = std::min<long long>(c, std::max<long long>(1, wmax / 2));
        c = std::max<long long>(1, std::min<long long>(c, cap));
        p.wave_off.push_back(static_cast<int>(p.wave_tiles.size()));
        p.wave_cnt.push_back(static_cast<int>(nt));
        p.wave_csize.push_back(static_cast<int>(c));
        p.wave_tiles.insert(p.wave_tiles.end(), v.begin(), v.end());
    }
    // executed flops: every block-update job is TE^(d+1) multiply-adds per
    // product (1 product Laplace; 2 / 3 / 2 for the generalized levels), the
    // generalized diagonal chain adds 3(d-2)+2 products per block, and the
    // base case costs one multiply-add per in-block line entry beyond the
    // diagonal and per product of the generalized recurrence.
    const double unit = 2.0 * p.td * p.te;
    double f = 0;
    for (long long t = 0; t < p.ntiles; t++) f += cost[t] * unit;
    if (p.gen && d >= 2) f += p.ntiles * (3.0 * (d - 2) + 2) * unit;
    if (p.tt) f += p.ntiles * (d - 1.0) * unit;  // the diagonal chain of the level sums
    double inblock = 0;
    for (int mu = 0; mu < d; mu++) inblock += (p.te - 1) / 2.0;
    f += p.ntiles * p.td * 2.0 * inblock * (p.gen ? (3.0 * d - 2) : p.tt ? 1.0 + (d - 1.0) : 1.0);
    p.flops = f;
}

}  // namespace

void fill_plan(Plan& p, int d, const long long* n, bool gen, int elem, int split, const std::vector<uint8_t>& sub,
               int partition, int shape, bool tt) {
    p.d = d;
    p.shape = shape;
    p.tt = tt && d >= 2;
    p.gen = gen && d >= 2;
    p.te = tile_extent(d);
    p.td = ipow(p.te, d);
    p.tc = p.te * p.te;
    p.elem = elem;
    size_t off = 0;
    long long ts = 1;
    for (int mu = 0; mu < d; mu++) {
        p.n[mu] = n[mu];
        std::vector<uint8_t> s(static_cast<size_t>(n[mu]), 0);
        for (long long i = 0; i + 1 < n[mu]; i++) s[i] = sub[off + i];
        off += static_cast<size_t>(n[mu] - 1);
        p.part[mu] = make_part(static_cast<int>(n[mu]), s, shape_cut(d, mu, shape), partition);
        p.nb[mu] = p.part[mu].nb;
        p.tstride[mu] = ts;
        ts *= p.nb[mu];
    }
    p.ntiles = ts;
    build_waves(p, split);
    // device tables
    p.tab.clear();
    for (int mu = 0; mu < d; mu++) {
        p.t_start[mu] = p.tab.size();
        p.tab.insert(p.tab.end(), p.part[mu].start.begin(), p.part[mu].start.end());
        p.t_size[mu] = p.tab.size();
        p.tab.insert(p.tab.end(), p.part[mu].size.begin(), p.part[mu].size.end());
        p.t_blk[mu] = p.tab.size();
        p.tab.insert(p.tab.end(), p.part[mu].blk_of.begin(), p.part[mu].blk_of.end());
    }
    p.t_wave = p.tab.size();
    p.tab.insert(p.tab.end(), p.wave_tiles.begin(), p.wave_tiles.end());
    if (elem == 4 && !p.gen && !p.tt && d >= 2 && p.ntiles < (1LL << 26)) {
        // S1, R1, S2, R2 of anti-diagonal w at virtual times w, w + lag,
        // w + 2 lag, w + 3 lag: every job comes after the jobs it waits for
        p.t_rjobs = p.tab.size();
        const int nw = static_cast<int>(p.wave_off.size());
        for (int tau = 0; tau < nw + 3 * kRefine2Lag; tau++)
            for (int kind = 0; kind < 4; kind++) {
                const int w = tau - kind * kRefine2Lag;
                if (w < 0 || w >= nw) continue;
                for (int i = 0; i < p.wave_cnt[w]; i++)
                    p.tab.push_back((kind << 26) | p.wave_tiles[p.wave_off[w] + i]);
            }
        p.n_rjobs = static_cast<int>(p.tab.size() - p.t_rjobs);
    }
}

std::shared_ptr<Plan> get_plan(int d, const long long* n, bool gen, int elem, int split,
                               const std::vector<uint8_t>* sub, int partition, int shape, bool tt) {
    std::string key = std::to_string(d) + (tt ? "w" : gen ? "g" : "l") + std::to_string(elem) + "s" +
                      std::to_string(split) + "p" + std::to_string(partition) + "t" + std::to_string(shape);
    size_t off = 0;
    for (int mu = 0; mu < d; mu++) {
        key += ":" + std::to_string(n[mu]) + ":";
        for (long long i = 0; i + 1 < n[mu]; i++) key += sub[0][off + i] ? '1' : '0';
        off += static_cast<size_t>(n[mu] - 1);
    }
    std::lock_guard<std::mutex> lk(g_mutex);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) return it->second;
    auto p = std::make_shared<Plan>();
    fill_plan(*p, d, n, gen, elem, split, *sub, partition, shape, tt);
    if (cudaMallocHost(&p->h_tab, p->tab.size() * sizeof(int)) != cudaSuccess) return nullptr;
    std::memcpy(p->h_tab, p->tab.data(), p->tab.size() * sizeof(int));
    g_plans[key] = p;
    return p;
}

GeomArgs geom_of(const Plan& p, const Layout& L, char* base, bool flip) {
    GeomArgs g{};
    g.d = p.d;
    const int* tab = reinterpret_cast<const int*>(base + L.tab);
    for (int mu = 0; mu < p.d; mu++) {
        g.n[mu] = p.n[mu];
        g.nb[mu] = p.nb[mu];
        g.tstride[mu] = p.tstride[mu];
        g.part.start[mu] = tab + p.t_start[mu];
        g.part.size[mu] = tab + p.t_size[mu];
        g.part.blk_of[mu] = tab + p.t_blk[mu];
    }
    g.ntiles = p.ntiles;
    g.flip = flip ? 1 : 0;
    return g;
}

}  // namespace tsylv
