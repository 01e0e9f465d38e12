// Host-side schedule: the split tree of Alg. 2 (Sec. 2.1) turned into a block
// grid, its wavefronts, the workspace layout and the captured CUDA graphs.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "tsylv_internal.h"

namespace tsylv {

// Partition of one mode into the leaves of the split tree.
struct Part {
    int n = 0;
    int nb = 0;
    std::vector<int> start, size, blk_of;
};

// The split rule of Alg. 2 applied recursively to one mode: split m at
// k = floor(m/2), k+1 when A(k+1, k) != 0 (1-based) so that no 2x2 block is
// cut, until every piece has at most te entries.  sub[i] != 0 marks A(i+1, i).
Part make_part(int n, const std::vector<uint8_t>& sub, int te, int rule);

// Largest number of leaves any admissible block structure can produce.
int max_blocks(int n, int te);

// Tile shapes: the leaf bound (the recursion cutoff n_min of the split tree)
// of every mode, at most the tile extent TE of the order d.  Candidates of
// the autotuner: 0 every mode TE; 1 every mode TE - 1; 2 every mode 3/4 TE;
// 3 every mode TE/2; 4 the last mode TE/2, the others TE (bounds at least 2).
// A shape id >= kShapeFixed holds fixed bounds (opts->nmin, opts->leaf): the
// bound of mode mu in bits 6 mu .. 6 mu + 5 of id - kShapeFixed, a zero field
// taking the bound of mode 1 (so id - kShapeFixed = c is the uniform bound c).
constexpr int kShapes = 5;
constexpr int kShapeFixed = 100;
int shape_cut(int d, int mu, int shape);
// Smallest bound of mode mu over the shapes a call may use (shape < 0: every
// candidate) -- the workspace bounds take it.
int shape_min_cut(int d, int mu, int shape);

struct GraphEntry {
    std::vector<const void*> key;
    cudaGraphExec_t exec = nullptr;
};

// One solve schedule: a block grid with its anti-diagonal wavefronts.
struct Plan {
    int d = 0, te = 0, td = 0, tc = 0;
    int shape = 0;                   // tile shape (leaf bound of every mode, shape_cut)
    bool gen = false;
    bool tt = false;                 // the two-term form Eq. (3.1)
    int elem = 8;                    // bytes per block-tensor entry
    long long n[kMaxD] = {};
    Part part[kMaxD];
    int nb[kMaxD] = {};
    long long tstride[kMaxD] = {};
    long long ntiles = 0;
    // wavefronts, highest anti-diagonal first
    std::vector<int> wave_tiles;
    std::vector<int> wave_off, wave_cnt, wave_csize;
    double flops = 0;                // executed flops of one solve
    // device tables (ints): start/size/blk_of per mode, then wave tiles
    std::vector<int> tab;
    size_t t_start[kMaxD] = {}, t_size[kMaxD] = {}, t_blk[kMaxD] = {}, t_wave = 0;
    // job queue of the pipelined first two refinement steps (FP32 Laplace
    // plans, d >= 2): kind << 26 | block, kinds S1, R1, S2, R2 of each
    // anti-diagonal kRefine2Lag anti-diagonals apart
    size_t t_rjobs = 0;
    int n_rjobs = 0;
    int* h_tab = nullptr;            // pinned copy of tab (source of the graph's upload)
    std::vector<GraphEntry> graphs;
    cudaEvent_t ev[4] = {};          // opts->timing: call start, waves begin/end, call end
    ~Plan();
};

constexpr int kRefine2Lag = 2;

// Workspace regions, as byte offsets from the (256-byte aligned) base.
struct Layout {
    size_t err = 0, sub = 0, tab = 0;
    size_t fargs = 0, fctl = 0, flags = 0;  // persistent schedule: parameter block, queue head + abort, solved flags
    size_t X = 0, P[kMaxD] = {}, G[kMaxD] = {}, At[kMaxD] = {}, Ct[kMaxD] = {};
    size_t total = 0;
};

// tt: the two-term form (stored intermediates Q_l in P, C tiles of mode 1 only).
Layout make_layout(int d, const long long* n, const int* nb, bool gen, int elem, size_t tab_ints, bool tt = false);

// Schedule of one solve (partition, wavefronts, device tables) without the
// pinned host copy of the tables and without caching.
void fill_plan(Plan& p, int d, const long long* n, bool gen, int elem, int split, const std::vector<uint8_t>& sub,
               int partition, int shape = 0, bool tt = false);

// Cached schedule with a pinned copy of its tables (the source of a captured upload).
std::shared_ptr<Plan> get_plan(int d, const long long* n, bool gen, int elem, int split,
                               const std::vector<uint8_t>* sub, int partition, int shape = 0, bool tt = false);

GeomArgs geom_of(const Plan& p, const Layout& L, char* base, bool flip);

}  // namespace tsylv
