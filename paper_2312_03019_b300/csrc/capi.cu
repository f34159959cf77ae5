// capi.cu -- host runtime behind include/qaoa.h.
//
// A state handle binds a caller-owned device buffer and stream to a graph.  qaoa_apply_layers
// uploads the levels' angles as kernel parameters, builds the per-level phase tables on the
// device (coeff_kernel), and enqueues the pass plan of plan.h: one tile_kernel launch per pass
// (n > Q_small) or one small_kernel launch for all levels (n <= Q_small).  The expectation is
// fused into the last pass; qaoa_expectation only reduces the per-tile partials.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <type_traits>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qaoa.h"
#include "kernels.cuh"
#include "instances.h"
#include "plan.h"

using namespace qaoa;

namespace {

thread_local std::string g_last_error;

qaoa_status fail(qaoa_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

qaoa_status cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return QAOA_ERR_CUDA;
}

#define CUDA_TRY(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

constexpr int kSmallMaxC64 = 14;   // 2^14 x 8 B = 128 KiB of shared memory
constexpr int kSmallMaxC128 = 13;  // 2^13 x 16 B

struct HostGraph {
    int n = 0, m = 0;
    std::vector<std::pair<int, int>> edges;  // u < v, ascending
    uint64_t upper[kMaxN] = {};              // graph_I rows (Table 1)
    uint64_t adj[kMaxN] = {};                // full adjacency
    bool weighted = false;                   // false: every weight is 1 (the cut count)
    std::vector<double> w;                   // weight of edges[e] (weighted graphs)
};

// Phase-table entries per level: |E| + 1 for the cut count; kWTurnSteps rotations of the folded
// factor when the phase comes from the weighted sums.
int table_entries(const HostGraph& g) { return g.weighted ? kWTurnSteps : g.m + 1; }

// 2^S for the value weights: the largest power of two with sum |w_e| 2^S <= 2^(B-2), B the
// fixed-point word size of the precision (32 for complex64, 64 for complex128), and S <= 1000 so
// that 2^S stays finite for the tiniest weights (those then round to zero, within the
// m 2^-(S+1) bound).
double value_mul(const HostGraph& g, int prec) {
    double tot = 0.0;
    for (double x : g.w) tot += std::fabs(x);
    const int B = prec == QAOA_C64 ? 32 : 64;
    if (!(tot > 0.0)) return std::ldexp(1.0, B - 2);
    return std::ldexp(1.0, std::min(1000, B - 2 - (int)std::ceil(std::log2(tot))));
}

qaoa_status encode_graph(const qaoa_graph* g, HostGraph& hg) {
    if (!g) return fail(QAOA_ERR_INVALID, "graph is NULL");
    if (g->n < 1 || g->n > kMaxN) return fail(QAOA_ERR_INVALID, "n must be in [1, 34]");
    if (g->m < 0) return fail(QAOA_ERR_INVALID, "m must be >= 0");
    if (g->m > 0 && !g->edges) return fail(QAOA_ERR_INVALID, "edges is NULL");
    hg.n = g->n;
    hg.m = g->m;
    std::set<std::pair<int, int>> seen;
    std::vector<std::pair<std::pair<int, int>, double>> ew;
    bool unit = true;
    for (int e = 0; e < g->m; ++e) {
        int u = g->edges[2 * e], v = g->edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= g->n || v >= g->n) return fail(QAOA_ERR_INVALID, "edge endpoint out of range");
        if (u == v) return fail(QAOA_ERR_INVALID, "self loop");
        if (u > v) std::swap(u, v);
        if (!seen.insert({u, v}).second) return fail(QAOA_ERR_INVALID, "repeated edge");
        const double w = g->weights ? g->weights[e] : 1.0;
        if (!std::isfinite(w)) return fail(QAOA_ERR_INVALID, "non-finite edge weight");
        if (std::fabs(w) > 1e12) return fail(QAOA_ERR_INVALID, "edge weight magnitude above 1e12");
        unit = unit && w == 1.0;
        ew.push_back({{u, v}, w});
        hg.upper[u] |= 1ull << v;
        hg.adj[u] |= 1ull << v;
        hg.adj[v] |= 1ull << u;
    }
    std::sort(ew.begin(), ew.end());
    for (const auto& x : ew) hg.edges.push_back(x.first);
    hg.weighted = !unit;  // all weights 1: the integer cut-count path, identical results
    if (hg.weighted)
        for (const auto& x : ew) hg.w.push_back(x.second);
    return QAOA_OK;
}

bool is_small(int n, int prec) { return n <= (prec == QAOA_C64 ? kSmallMaxC64 : kSmallMaxC128); }

size_t elem_bytes(int prec) { return prec == QAOA_C64 ? 8 : 16; }

// NVTX ranges (header-only NVTX 3): a profiler that records them (Nsight Systems, or ncu's
// --nvtx filters) sees each API call and each state pass by name; without one attached a push
// and a pop cost nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#ifdef QAOA_DEBUG_BOUNDS
// The index-check word of the debug build (see QAOA_IN_BOUNDS in kernels.cuh).  Host code only
// holds a stand-in for it: its device address is looked up once per device.
static __device__ unsigned int g_bounds_flag;
unsigned* bounds_flag_ptr() {
    static std::mutex mu;
    static std::vector<unsigned*> ptrs;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)ptrs.size() <= dev) ptrs.resize(dev + 1, nullptr);
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bounds_flag) == cudaSuccess) ptrs[dev] = static_cast<unsigned*>(p);
    }
    return ptrs[dev];
}
#else
unsigned* bounds_flag_ptr() { return nullptr; }
#endif

// Per-geometry decomposition tables of the on-the-fly cut count.
template <int Q>
void fill_geometry(TileArgs<Q>& a, const HostGraph& hg, const Geometry& geo, const TileConfig& tc) {
    a.n = hg.n;
    a.bounds_flag = bounds_flag_ptr();
    for (int v = 0; v < kMaxN; ++v) a.gmask[v] = v < hg.n ? hg.upper[v] : 0;
    int lpos[kMaxN];
    for (int w = 0; w < kMaxN; ++w) lpos[w] = -1;
    uint64_t tileMask = 0;
    for (int u = 0; u < Q; ++u) {
        lpos[geo.gpos[u]] = u;
        tileMask |= 1ull << geo.gpos[u];
    }
    // tile id bits -> outer index bits, as runs of consecutive positions (ascending)
    a.nruns = 0;
    int src = 0;
    for (int w = 0; w < hg.n;) {
        if (lpos[w] >= 0) {
            ++w;
            continue;
        }
        int len = 0;
        while (w + len < hg.n && lpos[w + len] < 0) ++len;
        a.run_src[a.nruns] = (uint8_t)src;
        a.run_len[a.nruns] = (uint8_t)len;
        a.run_dst[a.nruns] = (uint8_t)w;
        ++a.nruns;
        src += len;
        w += len;
    }
    // per register layout: index bits of the thread bits, strides and steps of the register bits
    const int R = tc.R;
    for (int L = 0; L < 3; ++L) {
        for (int k = 0; k < Q - R; ++k) {
            const int local = L == 0 ? k : (L == 1 ? (k < Q - 2 * R ? k : k + R) : k + R);
            a.tpos[L][k] = (uint8_t)geo.gpos[local];
        }
        int64_t below = 0;
        for (int j = 0; j < R; ++j) {
            const int64_t st = (int64_t)1 << geo.gpos[tc.regLo(L) + j];
            a.rstride[L][j] = st;
            a.rstep[L][j] = st - below;
            below += st;
        }
    }
    const uint64_t nMask = hg.n >= 64 ? ~0ull : ((1ull << hg.n) - 1ull);
    for (int u = 0; u < Q; ++u) {
        const int gu = geo.gpos[u];
        uint32_t la = 0;
        for (int w = 0; w < hg.n; ++w)
            if (((hg.adj[gu] >> w) & 1ull) && lpos[w] >= 0) la |= 1u << lpos[w];
        a.locAdj[u] = la;
        a.locUpper[u] = la & ~((2u << u) - 1u);
        a.outAdj[u] = hg.adj[gu] & ~tileMask & nMask;
    }
    // weighted split: local bit of every index bit and the tile-internal edges (edge-weighted
    // graphs only; the allocation-free path encodes unit-weight graphs without the edge list)
    a.m = hg.m;
    a.wn = 0;
    for (int v = 0; v < kMaxN; ++v) a.gl2loc[v] = (v < hg.n && lpos[v] >= 0) ? (uint8_t)lpos[v] : (uint8_t)0xff;
    for (int e = 0; hg.weighted && e < hg.m; ++e) {
        const int la = lpos[hg.edges[e].first], lb = lpos[hg.edges[e].second];
        if (la < 0 || lb < 0) continue;
        a.wloc[a.wn++] = (uint32_t)e | (uint32_t)std::min(la, lb) << 10 | (uint32_t)std::max(la, lb) << 14;
    }
    for (int L = 0; L < 3; ++L) {
        const int rl = tc.regLo(L);
        for (int x = 0; x < 32; ++x) {
            int c = 0;
            if (x < (1 << tc.R))
                for (int j = 0; j < tc.R; ++j)
                    for (int m = j + 1; m < tc.R; ++m)
                        if ((a.locAdj[rl + j] >> (rl + m)) & 1u) c += ((x >> j) ^ (x >> m)) & 1;
            a.crtab[L][x] = c;
        }
    }
}

// Weighted-sum slots of one pass: slot 0 is the value row (<C>, lambda, the gamma terms); each
// level whose phase the pass applies gets the next slot, reading wfix row 2 + level.
template <int Q>
bool fill_weighted(TileArgs<Q>& a, const HostGraph& g, int prec, const void* wfix, const Op* ops, int nops) {
    a.wfix = wfix;
    a.vscale = 1.0 / value_mul(g, prec);
    a.wrow[0] = 1;
    a.wnslots = 1;
    for (int i = 0; i < nops; ++i) {
        if (ops[i].kind != OP_PHASE && ops[i].kind != OP_PHASED) continue;
        const int level = ops[i].arg & 0xffff;
        bool have = false;
        for (int sl = 1; sl < a.wnslots; ++sl) have = have || a.wrow[sl] == 2 + level;
        if (have) continue;
        if (a.wnslots == kWSlots || level >= kLayerChunk) return false;
        a.wslot[level] = (int8_t)a.wnslots;
        a.wrow[a.wnslots++] = (int16_t)(2 + level);
    }
    return true;
}

// Weights, endpoints and the value scale of an edge-weighted graph in the coefficient launch.
void fill_coeff_weights(CoeffArgs& ca, const HostGraph& g, int prec, void* wfix, int wrow0) {
    if (!g.weighted) return;
    ca.weighted = 1;
    ca.m = g.m;
    ca.wrow0 = wrow0;
    ca.vmul = value_mul(g, prec);
    ca.wfix = wfix;
    for (int e = 0; e < g.m; ++e) {
        ca.w[e] = g.w[e];
        ca.uv[e] = (uint16_t)(g.edges[e].first | g.edges[e].second << 8);
    }
}

// Device bytes of the fixed-point rows: endpoints, values and `levels` angle rows.
size_t wfix_bytes(const HostGraph& g, int prec, int levels) {
    return (size_t)(2 + levels) * (size_t)std::max(1, g.m) * (prec == QAOA_C64 ? 4 : 8);
}

template <typename J>
void set_small_weights(J& j, const HostGraph& g, int prec, const void* wfix) {
    if (!g.weighted) return;
    j.wfix = wfix;
    j.m = g.m;
    j.vscale = 1.0 / value_mul(g, prec);
}

template <typename real>
struct PrecTraits;
template <>
struct PrecTraits<float> {
    static constexpr int Q = 13, R = 5;
};
template <>
struct PrecTraits<double> {
    static constexpr int Q = 12, R = 4;
};

// Tiles of the adjoint sweep: Q = 12, R = 4 in both precisions (the sweep holds psi and lambda,
// two 16-amplitude register sets per thread, so two CTAs fit per SM in complex64).
template <typename real>
struct GradTraits {
    static constexpr int Q = 12, R = 4;
};

TileConfig grad_tile_config(int prec) {
    if (prec == QAOA_C64) return TileConfig{12, 4, 3, 18};  // 64-byte rows, 2 MiB pages of complex64
    return tile_config_for(prec);
}

uint64_t grad_tiles(int n) { return n > 12 ? 1ull << (n - 12) : 1ull; }

// Adjoint passes whose per-tile partials are reduced together (grad_reduce_batch_kernel): as many
// as 32 MiB of partials hold, at most kGradBatchMax and at most the 3p + 1 passes a sweep of p
// levels can have (non-decreasing in p, so workspace sized for p serves any smaller p).
int grad_chunk(int n, int p) {
    const uint64_t per_pass = 2 * grad_tiles(n) * sizeof(double2);
    const uint64_t fit = std::max<uint64_t>(1, (32ull << 20) / per_pass);
    return (int)std::min<uint64_t>({fit, (uint64_t)kGradBatchMax, (uint64_t)(3 * p + 1)});
}
size_t grad_partials_bytes(int n, int p) { return (size_t)grad_chunk(n, p) * 2 * grad_tiles(n) * sizeof(double2); }
// Per-level sums [2p], the batch sums [4 kGradBatchMax] and the batch ticket.
size_t grad_acc_bytes(int p) { return ((size_t)2 * p + 4 * kGradBatchMax + 1) * sizeof(double); }

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    // 1 read+write mixer-only pass, 2 synthesising pass, 3 read+write pass with a cost phase,
    // 4 read+write pass with <C>
    int kind = 0;
};

}  // namespace

struct qaoa_state_s {
    int dev = 0;
    int n = 0;
    int prec = 0;
    uint64_t dim = 0;
    void* buf = nullptr;
    cudaStream_t stream = nullptr;
    HostGraph g;
    TileConfig tc{};
    std::vector<Group> groups;
    bool small = false;
    uint64_t ntiles = 1;
    void* d_phase = nullptr;
    void* d_mix = nullptr;
    void* d_wfix = nullptr;       // weighted graphs: fixed-point rows (2 + kLayerChunk) x m
    void* d_gwfix = nullptr;      // weighted graphs: the adjoint sweep's rows (2 + levels) x m
    double2* d_partials = nullptr;
    double2* d_result = nullptr;
    double2 h_result[1] = {};     // <C> and norm read back (pageable: the read synchronises anyway)
    uint64_t partial_count = 0;
    void* ws = nullptr;           // the block d_phase .. d_result are carved from (library pool)
    void* gws = nullptr;          // the block of the adjoint sweep's workspace (library pool)
    // adjoint sweep workspace (allocated on the first qaoa_gradient call, grown as needed)
    int grad_levels = 0;
    void* d_gtab = nullptr;       // plain phase tables, [level][E1]
    void* d_gmix = nullptr;       // [3 * level] mixer entries
    double* d_gacc = nullptr;     // [2 * levels]
    double2* d_gpart = nullptr;   // [grad_chunk passes][2 * tiles]
    double* d_gpow = nullptr;     // complex64 sweep: [level][kMaxN + 1] powers of the butterflies' factor
    bool lazy = true;
    bool exp_valid = false;
    bool compl_ = false;  // buffer index z holds the amplitude of ~z (pending X on every qubit)
    bool pform_ = false;  // complex64 parity form: odd-parity indices hold (im, re)
    // profiling
    bool prof = false;
    std::vector<EventPair> events;
    size_t ev_used = 0;
    int64_t launches = 0;
};

namespace {

EventPair* next_event(qaoa_state s, int kind) {
    if (!s->prof) return nullptr;
    if (s->ev_used == s->events.size()) {
        EventPair p;
        if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return nullptr;
        s->events.push_back(p);
    }
    EventPair* e = &s->events[s->ev_used++];
    e->kind = kind;
    return e;
}

// Dynamic shared-memory limits of the kernels, set once per process (first use, or by
// prepare_kernels before any stream capture).
template <typename real>
using TileFn = void (*)(TileArgs<PrecTraits<real>::Q>);

// The straight-line instantiation of recipe r (unit weights).
template <typename real, int r, bool kW = false>
constexpr TileFn<real> recipe_fn() {
    return tile_kernel<real, PrecTraits<real>::Q, PrecTraits<real>::R, kW, recipe_def(r).code, recipe_def(r).nops,
                       recipe_masks<real>(r), recipe_def(r).hi>;
}

// The weighted (complex64) instantiation of recipe r, or NULL where none is compiled.
template <typename real>
TileFn<real> recipe_kernel_w(int r) {
    if constexpr (std::is_same<real, float>::value) {
        switch (r) {
            case 0: return recipe_fn<real, 0, true>();
            case 2: return recipe_fn<real, 2, true>();
            case 3: return recipe_fn<real, 3, true>();
            case 5: return recipe_fn<real, 5, true>();
            case 7: return recipe_fn<real, 7, true>();
            default: return nullptr;
        }
    }
    return nullptr;
}

// The unit-weight instantiation of recipe r, or NULL where none is compiled (the two-group
// programs 8..12 exist for complex64 only).
template <typename real>
TileFn<real> recipe_kernel(int r) {
    if constexpr (std::is_same<real, float>::value) {
        switch (r) {
            case 8: return recipe_fn<real, 8>();
            case 9: return recipe_fn<real, 9>();
            case 10: return recipe_fn<real, 10>();
            case 11: return recipe_fn<real, 11>();
            case 12: return recipe_fn<real, 12>();
            default: break;
        }
    }
    if (r >= 8) return nullptr;
    switch (r) {
        case 0: return recipe_fn<real, 0>();
        case 1: return recipe_fn<real, 1>();
        case 2: return recipe_fn<real, 2>();
        case 3: return recipe_fn<real, 3>();
        case 4: return recipe_fn<real, 4>();
        case 5: return recipe_fn<real, 5>();
        case 6: return recipe_fn<real, 6>();
        default: return recipe_fn<real, 7>();
    }
}

// The compiled recipe a program runs, or -1 for the interpreting instantiation: the first recipe
// (those with compiled-in masks first, and only when the program's masks are exactly those) whose
// ops and layouts equal the program's and which is compiled for this precision and weighting.
// Edge weights enter only the phase, <C> and cut-value ops: a program without them (a plain mixer
// pass) runs the unit-weight instance, whatever the graph.
template <typename real>
int pick_recipe(const TileArgs<PrecTraits<real>::Q>& a, bool weighted_graph) {
    const bool weighted = weighted_graph && a.need_cut;
    if (a.nops > 20) return -1;
    uint64_t code = 0, hi = 0;
    for (int i = 0; i < a.nops; ++i) {
        code |= recipe_step_lo(i, a.ops[i].kind, a.ops[i].layout);
        hi |= recipe_step_hi(i, a.ops[i].kind, a.ops[i].layout);
    }
    // full-mask instantiations first (5, 6, 7), then the runtime-mask ones
    const int order[] = {1, 5, 6, 7, 0, 2, 3, 4, 8, 9, 10, 11, 12};
    for (int r : order) {
        const Recipe d = recipe_def(r);
        if (d.nops != a.nops || d.code != code || d.hi != hi) continue;
        bool masks_ok = true;
        for (int i = 0; i < a.nops && i < 10; ++i) {
            const uint32_t fm = (uint32_t)((recipe_masks<real>(r) >> (6 * i)) & 63u);
            if ((fm & 32u) && a.ops[i].mask != (fm & 31u)) masks_ok = false;
        }
        if (!masks_ok) continue;
        if (weighted ? recipe_kernel_w<real>(r) != nullptr : recipe_kernel<real>(r) != nullptr) return r;
    }
    return -1;
}

// The pass kernel for a program: its recipe instantiation, else the interpreting one.
template <typename real>
TileFn<real> pick_tile_kernel(const TileArgs<PrecTraits<real>::Q>& a, bool weighted_graph) {
    constexpr int Q = PrecTraits<real>::Q, R = PrecTraits<real>::R;
    const bool weighted = weighted_graph && a.need_cut;
    const int r = pick_recipe<real>(a, weighted_graph);
    if (r >= 0) return weighted ? recipe_kernel_w<real>(r) : recipe_kernel<real>(r);
    return weighted ? tile_kernel<real, Q, R, true> : tile_kernel<real, Q, R, false>;
}

// The packed (tile_batch_kernel) form of the kernel pick_tile_kernel gives a unit-weight
// complex64 program, for the programs of the two-group plans (recipes 8..12 or the interpreting
// instance); NULL for others, which then run alone.
template <typename real>
using TileBatchFn = void (*)(const TileArgs<PrecTraits<real>::Q>*);

template <typename real, int r>
constexpr TileBatchFn<real> batch_recipe_fn() {
    return tile_batch_kernel<real, PrecTraits<real>::Q, PrecTraits<real>::R, false, recipe_def(r).code,
                             recipe_def(r).nops, recipe_masks<real>(r), recipe_def(r).hi>;
}

template <typename real>
TileBatchFn<real> batch_kernel_for(int r) {
    if constexpr (std::is_same<real, float>::value) {
        switch (r) {
            case -1: return tile_batch_kernel<real, PrecTraits<real>::Q, PrecTraits<real>::R, false>;
            case 8: return batch_recipe_fn<real, 8>();
            case 9: return batch_recipe_fn<real, 9>();
            case 10: return batch_recipe_fn<real, 10>();
            case 11: return batch_recipe_fn<real, 11>();
            case 12: return batch_recipe_fn<real, 12>();
            default: return nullptr;
        }
    }
    return nullptr;
}

template <typename real>
TileBatchFn<real> pick_tile_batch_kernel(const TileArgs<PrecTraits<real>::Q>& a) {
    return batch_kernel_for<real>(pick_recipe<real>(a, false));
}

template <typename real>
using GradFn = void (*)(TileArgs<GradTraits<real>::Q>);

// The straight-line adjoint-pass instantiation of sweep program r (complex64) with the RXD masks
// of variant v compiled in (grad_masks; v = 0: runtime masks).
template <int r, bool kW, int v = 0>
constexpr GradFn<float> grad_recipe_fn() {
    return grad_kernel<float, GradTraits<float>::Q, GradTraits<float>::R, kW, grad_recipe(r).code,
                       grad_recipe(r).nops, grad_masks(r, v)>;
}
template <bool kW>
GradFn<float> grad_recipe_fn_for(int r, int v) {
    if (r == 0) return v == 1 ? grad_recipe_fn<0, kW, 1>() : v == 0 ? grad_recipe_fn<0, kW>() : nullptr;
    if (r == 1)
        return v == 1   ? grad_recipe_fn<1, kW, 1>()
               : v == 2 ? grad_recipe_fn<1, kW, 2>()
               : v == 3 ? grad_recipe_fn<1, kW, 3>()
                        : grad_recipe_fn<1, kW>();
    if (r == 3) return v == 1 ? grad_recipe_fn<3, kW, 1>() : v == 0 ? grad_recipe_fn<3, kW>() : nullptr;
    if (r == 4) return v == 1 ? grad_recipe_fn<4, kW, 1>() : v == 0 ? grad_recipe_fn<4, kW>() : nullptr;
    if (r == 2) return v == 0 ? grad_recipe_fn<2, kW>() : nullptr;
    return nullptr;  // programs 5..8: persistent form only
}
template <typename real>
GradFn<real> grad_recipe_kernel(int r, bool weighted, int v = 0) {
    if constexpr (std::is_same<real, float>::value)
        return weighted ? grad_recipe_fn_for<true>(r, v) : grad_recipe_fn_for<false>(r, v);
    return nullptr;
}

// The persistent prefetching form of compiled sweep program r with mask variant v (complex64,
// unit or edge weights; grad_pf_kernel), or nullptr.
using GradPfFn = void (*)(TileArgs<GradTraits<float>::Q>, uint64_t);
template <bool kW, int r, int v>
constexpr GradPfFn grad_pf_fn() {
    return grad_pf_kernel<GradTraits<float>::Q, GradTraits<float>::R, kW, grad_recipe(r).code, grad_recipe(r).nops,
                          grad_masks(r, v), grad_recipe(r).hi>;
}
template <bool kW>
GradPfFn grad_pf_for_w(int r, int v) {
    switch (r * 8 + v) {
        case 0 * 8 + 1: return grad_pf_fn<kW, 0, 1>();
        case 1 * 8 + 0: return grad_pf_fn<kW, 1, 0>();
        case 1 * 8 + 1: return grad_pf_fn<kW, 1, 1>();
        case 1 * 8 + 2: return grad_pf_fn<kW, 1, 2>();
        case 1 * 8 + 3: return grad_pf_fn<kW, 1, 3>();
        case 3 * 8 + 0: return grad_pf_fn<kW, 3, 0>();
        case 3 * 8 + 1: return grad_pf_fn<kW, 3, 1>();
        case 4 * 8 + 0: return grad_pf_fn<kW, 4, 0>();
        case 4 * 8 + 1: return grad_pf_fn<kW, 4, 1>();
        case 5 * 8 + 0: return grad_pf_fn<kW, 5, 0>();
        case 6 * 8 + 0: return grad_pf_fn<kW, 6, 0>();
        case 7 * 8 + 0: return grad_pf_fn<kW, 7, 0>();
        case 8 * 8 + 0: return grad_pf_fn<kW, 8, 0>();
        default: return nullptr;
    }
}
GradPfFn grad_pf_for(int r, int v, bool weighted) {
    return weighted ? grad_pf_for_w<true>(r, v) : grad_pf_for_w<false>(r, v);
}

// The compiled sweep program (r, v) a pass's program matches, among those `exists(r, v)`
// accepts: the mask variants whose compiled-in masks are this pass's first, then the runtime
// one.  False: none (interpreting).
template <typename real, typename Exists>
bool match_grad_recipe(const TileArgs<GradTraits<real>::Q>& a, Exists&& exists, int* r_out, int* v_out) {
    if (!std::is_same<real, float>::value || a.nops > 20) return false;
    uint64_t lo = 0, hi = 0;
    for (int i = 0; i < a.nops; ++i) {
        lo |= recipe_step_lo(i, a.ops[i].kind, a.ops[i].layout);
        hi |= recipe_step_hi(i, a.ops[i].kind, a.ops[i].layout);
    }
    for (int r = 0; r < kGradRecipes; ++r) {
        const Recipe d = grad_recipe(r);
        if (d.nops != a.nops || d.code != lo || d.hi != hi) continue;
        for (int v = kGradMaskVariants - 1; v >= 0; --v) {
            const uint64_t m = grad_masks(r, v);
            if (v > 0 && m == 0) continue;
            bool ok = true;
            for (int i = 0; i < a.nops && i < 10; ++i) {
                const uint32_t fm = (uint32_t)((m >> (6 * i)) & 63u);
                if ((fm & 32u) && a.ops[i].mask != (fm & 31u)) ok = false;
            }
            if (!ok || !exists(r, v)) continue;
            *r_out = r;
            *v_out = v;
            return true;
        }
    }
    return false;
}

// The adjoint-pass kernel for a program: a compiled sweep program when one matches (complex64,
// unit or edge weights), else the interpreting instantiation.
template <typename real>
GradFn<real> pick_grad_kernel(const TileArgs<GradTraits<real>::Q>& a, bool weighted) {
    constexpr int Q = GradTraits<real>::Q, R = GradTraits<real>::R;
    int r = 0, v = 0;
    auto exists = [&](int rr, int vv) { return grad_recipe_kernel<real>(rr, weighted, vv) != nullptr; };
    if (match_grad_recipe<real>(a, exists, &r, &v))
        if (GradFn<real> f = grad_recipe_kernel<real>(r, weighted, v)) return f;
    return weighted ? grad_kernel<real, Q, R, true> : grad_kernel<real, Q, R, false>;
}

// The persistent prefetching kernel for a pass, when its program has one (complex64, a compiled
// program with an exchange), else nullptr.
template <typename real>
GradPfFn pick_grad_pf_kernel(const TileArgs<GradTraits<real>::Q>& a, bool weighted) {
    int r = 0, v = 0;
    auto exists = [&](int rr, int vv) { return grad_pf_for(rr, vv, weighted) != nullptr; };
    if (!match_grad_recipe<real>(a, exists, &r, &v)) return nullptr;
    return grad_pf_for(r, v, weighted);
}

// CTAs of a persistent kernel that fit the current device at once (cached per device and kernel).
template <typename F>
unsigned resident_ctas(F f, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, unsigned> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, reinterpret_cast<const void*>(f));
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const unsigned n = (unsigned)std::max(0, per_sm * sms);
    cache[key] = n;
    return n;
}

// Dynamic shared-memory limits of every kernel, set once per device (the attribute belongs to
// the device's instance of the function) and thread-safely (the server's scheduler thread and
// callers' threads both launch).
template <typename real>
qaoa_status ensure_attributes() {
    static std::mutex mu;
    static std::vector<char> done;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < (int)done.size() && done[dev]) return QAOA_OK;
    constexpr int Q = PrecTraits<real>::Q, R = PrecTraits<real>::R;
    using C2 = typename C2T<real>::type;
    CUDA_TRY(cudaFuncSetAttribute(tile_kernel<real, Q, R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((1u << Q) * sizeof(C2))));
    CUDA_TRY(cudaFuncSetAttribute(tile_kernel<real, Q, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((1u << Q) * sizeof(C2))));
    for (int r = 0; r < kRecipes; ++r) {
        if (TileFn<real> f = recipe_kernel<real>(r))
            CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((1u << Q) * sizeof(C2))));
        if (TileFn<real> f = recipe_kernel_w<real>(r))
            CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((1u << Q) * sizeof(C2))));
    }
    for (int r : {-1, 8, 9, 10, 11, 12})
        if (TileBatchFn<real> f = batch_kernel_for<real>(r))
            CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((1u << Q) * sizeof(C2))));
    constexpr int GQ = GradTraits<real>::Q, GR = GradTraits<real>::R;
    // the adjoint passes exchange psi and lambda through a tile each
    CUDA_TRY(cudaFuncSetAttribute(grad_kernel<real, GQ, GR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * (1u << GQ) * sizeof(C2))));
    CUDA_TRY(cudaFuncSetAttribute(grad_kernel<real, GQ, GR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * (1u << GQ) * sizeof(C2))));
    if constexpr (std::is_same<real, float>::value)
        for (int r = 0; r < kGradRecipes; ++r)
            for (int v = 0; v < kGradMaskVariants; ++v) {
                for (bool w : {false, true})
                    if (GradFn<real> f = grad_recipe_kernel<real>(r, w, v))
                        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)(2 * (1u << GQ) * sizeof(C2))));
                for (bool w : {false, true})
                    if (GradPfFn f = grad_pf_for(r, v, w))
                        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)(2 * (1u << GQ) * sizeof(C2))));
            }
    CUDA_TRY(cudaFuncSetAttribute(small_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
    CUDA_TRY(cudaFuncSetAttribute(small_batch_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
    CUDA_TRY(cudaFuncSetAttribute(small_grad_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * (1u << Q) * sizeof(C2))));
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    done[dev] = 1;
    return QAOA_OK;
}

template <typename real>
qaoa_status prepare_kernels() {
    return ensure_attributes<real>();
}

template <typename real>
qaoa_status launch_tile(qaoa_state s, TileArgs<PrecTraits<real>::Q>& a, int kind) {
    constexpr int Q = PrecTraits<real>::Q, R = PrecTraits<real>::R;
    using C2 = typename C2T<real>::type;
    auto kfn = pick_tile_kernel<real>(a, s->g.weighted);
    const size_t smem = (size_t)(1u << Q) * sizeof(C2);
    qaoa_status ast = ensure_attributes<real>();
    if (ast != QAOA_OK) return ast;
    EventPair* ev = kind ? next_event(s, kind) : nullptr;
    if (ev) CUDA_TRY(cudaEventRecord(ev->a, s->stream));
    kfn<<<(unsigned)s->ntiles, 1u << (Q - R), smem, s->stream>>>(a);
    CUDA_TRY(cudaGetLastError());
    if (ev) CUDA_TRY(cudaEventRecord(ev->b, s->stream));
    s->launches++;
    return QAOA_OK;
}

template <typename real>
qaoa_status launch_small(qaoa_state s, const SmallJob& j) {
    using C2 = typename C2T<real>::type;
    auto kfn = small_kernel<real>;
    const size_t smem = (size_t)s->dim * sizeof(C2);
    qaoa_status ast = ensure_attributes<real>();
    if (ast != QAOA_OK) return ast;
    kfn<<<1, kSmallThreads, smem, s->stream>>>(j);
    CUDA_TRY(cudaGetLastError());
    s->launches++;
    return QAOA_OK;
}

// Pass arguments for the tile geometry of `groups[ps.group]` under tile configuration tc.
template <int Qt>
void fill_program_with(TileArgs<Qt>& a, qaoa_state s, const Pass& ps, const std::vector<Group>& groups,
                       const TileConfig& tc) {
    const Geometry geo = group_geometry(groups[ps.group], tc);
    fill_geometry(a, s->g, geo, tc);
    a.nops = (int)ps.ops.size();
    a.need_cut = 0;
    for (size_t i = 0; i < ps.ops.size(); ++i) {
        a.ops[i] = ps.ops[i];
        const uint8_t k = ps.ops[i].kind;
        if (k == OP_PHASE || k == OP_EXPECT || k == OP_CUTVAL) a.need_cut = 1;
    }
    a.E1 = table_entries(s->g);
    a.init_amp = std::pow(2.0, -0.5 * s->n);
    a.state = s->buf;
    a.phase = s->d_phase;
    a.mix = s->d_mix;
    a.partials = s->d_partials;
    a.cutout = nullptr;
    if (s->g.weighted) fill_weighted(a, s->g, s->prec, s->d_wfix, a.ops, a.nops);
}

template <typename real>
void fill_program(TileArgs<PrecTraits<real>::Q>& a, qaoa_state s, const Pass& ps) {
    fill_program_with(a, s, ps, s->groups, s->tc);
}

template <typename real>
qaoa_status run_plan(qaoa_state s, const Plan& plan) {
    constexpr int Q = PrecTraits<real>::Q;
    TileArgs<Q> a;
    for (const Pass& ps : plan.passes) {
        std::memset(&a, 0, sizeof(a));
        fill_program<real>(a, s, ps);
        int kind = 0;
        if (ps.store) {
            kind = ps.synth ? 2 : 1;
            for (int i = 0; kind == 1 && i < a.nops; ++i) {
                if (a.ops[i].kind == OP_PHASE) kind = 3;
                if (a.ops[i].kind == OP_EXPECT) kind = 4;
            }
        }
        static const char* const kPassName[] = {"qaoa pass (read only)", "qaoa pass (mixer)",
                                                "qaoa pass (first, synthesised)", "qaoa pass (fused, cost phase)",
                                                "qaoa pass (last, <C>)"};
        NvtxRange range(kPassName[kind]);
        qaoa_status st = launch_tile<real>(s, a, kind);
        if (st != QAOA_OK) return st;
    }
    return QAOA_OK;
}

template <typename real>
qaoa_status set_parity_form(qaoa_state s, bool parity);

// Coefficient arguments of one chunk of levels of state s (phase tables and mixer entries into
// s->d_phase / s->d_mix).  Returns whether the chunk leaves an odd number of folded levels, i.e.
// toggles the pending complement.
bool chunk_coeff_args(const qaoa_state_s* s, int levels, const double* gamma, const double* beta, CoeffArgs& ca) {
    std::memset(&ca, 0, sizeof(ca));
    ca.levels = levels;
    ca.E1 = table_entries(s->g);
    ca.n = s->n;
    ca.fold_factors = s->small ? 0 : 1;
    fill_coeff_weights(ca, s->g, s->prec, s->d_wfix, 2);
    int folded = 0;
    for (int k = 0; k < levels; ++k) {
        ca.gamma[k] = gamma[k];
        ca.beta[k] = beta[k];
        // Tile passes use RX(2b) = -i X RX(2b - pi) when |tan b| > 1, so that every butterfly
        // coefficient has |t| <= 1.  X on every qubit maps index z to ~z; it commutes with the
        // cost phase (C(~z) = C(z)) and the mixer, so it is only recorded (compl_).  The factors
        // (-i)^n are folded exactly into the last phase table of the chunk.
        ca.fold[k] = (!s->small && std::fabs(std::sin(beta[k])) > std::fabs(std::cos(beta[k]))) ? 1 : 0;
        folded += ca.fold[k];
    }
    const int quarter = (int)(((int64_t)folded * s->n) % 4);  // (-i)^quarter
    ca.gre = quarter == 0 ? 1 : (quarter == 2 ? -1 : 0);
    ca.gim = quarter == 1 ? -1 : (quarter == 3 ? 1 : 0);
    ca.phase = s->d_phase;
    ca.mix = s->d_mix;
    return (folded & 1) != 0;
}

dim3 coeff_grid(const CoeffArgs& ca) {
    return dim3((unsigned)std::max(1, (std::max(ca.E1, ca.m) + 255) / 256), (unsigned)std::max(1, ca.levels));
}

template <typename real>
qaoa_status apply_chunk(qaoa_state s, int levels, const double* gamma, const double* beta, bool expect) {
    CoeffArgs ca;
    if (chunk_coeff_args(s, levels, gamma, beta, ca)) s->compl_ = !s->compl_;
    dim3 grid = coeff_grid(ca);
    coeff_kernel<real><<<grid, 256, 0, s->stream>>>(ca);
    CUDA_TRY(cudaGetLastError());
    s->launches++;

    if (s->small) {
        SmallJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = s->n;
        j.levels = levels;
        j.E1 = table_entries(s->g);
        j.synth = s->lazy ? 1 : 0;
        j.expect = expect ? 1 : 0;
        j.store = 1;
        j.init_amp = std::pow(2.0, -0.5 * s->n);
        for (int v = 0; v < kMaxN; ++v) j.gmask[v] = v < s->n ? s->g.upper[v] : 0;
        j.state = s->buf;
        j.phase = s->d_phase;
        j.mix = s->d_mix;
        j.partials = s->d_partials;
        set_small_weights(j, s->g, s->prec, s->d_wfix);
        qaoa_status st = launch_small<real>(s, j);
        if (st != QAOA_OK) return st;
    } else {
        qaoa_status st = set_parity_form<real>(s, true);  // the passes read and write the parity form
        if (st != QAOA_OK) return st;
        Plan plan = plan_levels(s->n, s->tc, levels, s->lazy, expect);
        st = run_plan<real>(s, plan);
        if (st != QAOA_OK) return st;
        s->pform_ = std::is_same<real, float>::value;
    }
    s->lazy = false;
    if (expect) {
        s->exp_valid = true;
        s->partial_count = s->small ? 1 : s->ntiles;
    } else {
        s->exp_valid = false;
    }
    return QAOA_OK;
}

// Endpoint and value rows of an edge-weighted graph (a coefficient launch with no levels).
template <typename real>
qaoa_status write_weight_rows(qaoa_state s) {
    CoeffArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.levels = 0;
    ca.E1 = 1;
    ca.n = s->n;
    fill_coeff_weights(ca, s->g, s->prec, s->d_wfix, 2);
    coeff_kernel<real><<<(unsigned)std::max(1, (ca.m + 255) / 256), 256, 0, s->stream>>>(ca);
    CUDA_TRY(cudaGetLastError());
    s->launches++;
    return QAOA_OK;
}

template <typename real>
qaoa_status materialize(qaoa_state s) {
    if (s->lazy) {
        fill_kernel<real><<<148 * 8, 256, 0, s->stream>>>(s->buf, s->dim, std::pow(2.0, -0.5 * s->n));
        CUDA_TRY(cudaGetLastError());
        s->launches++;
        s->lazy = false;
        s->compl_ = false;  // |+>^n is its own complement
        s->pform_ = false;
    }
    if (s->compl_ || s->pform_) {
        complement_kernel<real><<<148 * 8, 256, 0, s->stream>>>(s->buf, s->dim, s->compl_ ? 1 : 0, s->pform_ ? 1 : 0);
        CUDA_TRY(cudaGetLastError());
        s->launches++;
        s->compl_ = false;
        s->pform_ = false;
    }
    return QAOA_OK;
}

// Puts (parity = true) or takes (false) the state buffer into / out of the complex64 parity form
// the forward tile passes keep it in between passes.
template <typename real>
qaoa_status set_parity_form(qaoa_state s, bool parity) {
    if (!std::is_same<real, float>::value || s->lazy || s->pform_ == parity) return QAOA_OK;
    complement_kernel<real><<<148 * 8, 256, 0, s->stream>>>(s->buf, s->dim, 0, 1);
    CUDA_TRY(cudaGetLastError());
    s->launches++;
    s->pform_ = parity;
    return QAOA_OK;
}

template <typename real>
qaoa_status compute_partials(qaoa_state s) {
    if (s->exp_valid) return QAOA_OK;
    if (s->small) {
        SmallJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = s->n;
        j.levels = 0;
        j.E1 = table_entries(s->g);
        j.synth = s->lazy ? 1 : 0;
        j.expect = 1;
        j.store = 0;
        j.init_amp = std::pow(2.0, -0.5 * s->n);
        for (int v = 0; v < kMaxN; ++v) j.gmask[v] = v < s->n ? s->g.upper[v] : 0;
        j.state = s->buf;
        j.phase = s->d_phase;
        j.mix = s->d_mix;
        j.partials = s->d_partials;
        set_small_weights(j, s->g, s->prec, s->d_wfix);
        qaoa_status st = launch_small<real>(s, j);
        if (st != QAOA_OK) return st;
        s->partial_count = 1;
    } else {
        Plan plan = plan_readonly(s->n, s->tc, s->lazy, OP_EXPECT, 0, 0);
        qaoa_status st = run_plan<real>(s, plan);
        if (st != QAOA_OK) return st;
        s->partial_count = s->ntiles;
    }
    s->exp_valid = true;
    return QAOA_OK;
}

// Enqueues the <C> / norm reduction of the current state into s->d_result (no host sync).
template <typename real>
qaoa_status expectation_async(qaoa_state s) {
    qaoa_status st = compute_partials<real>(s);
    if (st != QAOA_OK) return st;
    finalize_kernel<<<1, 1024, 0, s->stream>>>(s->d_partials, s->partial_count, s->d_result);
    CUDA_TRY(cudaGetLastError());
    s->launches++;
    return QAOA_OK;
}

template <typename real>
qaoa_status expectation_impl(qaoa_state s, double* out_c, double* out_norm) {
    qaoa_status st = expectation_async<real>(s);
    if (st != QAOA_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(s->h_result, s->d_result, sizeof(double2), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (out_c) *out_c = s->h_result->x;
    if (out_norm) *out_norm = s->h_result->y;
    return QAOA_OK;
}

// Per-state workspace comes from one stream-ordered memory pool per device, owned by the
// library: a state takes one block at qaoa_state_init (and one more at its first gradient) and
// gives it back at qaoa_state_free, on its own stream.  Freed blocks stay in the pool (up to
// kPoolKeepBytes per device) for the next state, so creating and freeing a state costs no
// cudaMalloc, cudaFree or device-wide synchronisation once the pool is warm.
constexpr uint64_t kPoolKeepBytes = 256ull << 20;

cudaError_t pool_create(int dev, cudaMemPool_t* out) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(out, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    return cudaMemPoolSetAttribute(*out, cudaMemPoolAttrReleaseThreshold, &keep);
}

// One block of `bytes` on `stream` from the pool of device `dev`.  A pool whose context is gone
// (after cudaDeviceReset) fails with an error other than out-of-memory: it is then created anew
// once.
cudaError_t ws_alloc(int dev, cudaStream_t stream, size_t bytes, void** out) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (!pools[dev]) {
            e = pool_create(dev, &pools[dev]);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
        }
        e = cudaMallocFromPoolAsync(out, bytes, pools[dev], stream);
        if (e == cudaSuccess || e == cudaErrorMemoryAllocation) return e;
        cudaGetLastError();
        pools[dev] = nullptr;
    }
    return e;
}

size_t ws_round(size_t x) { return (x + 255) & ~(size_t)255; }

void release(qaoa_state s) {
    if (!s) return;
    cudaSetDevice(s->dev);
    for (auto& e : s->events) {
        if (e.a) cudaEventDestroy(e.a);
        if (e.b) cudaEventDestroy(e.b);
    }
    if (s->ws) cudaFreeAsync(s->ws, s->stream);
    if (s->gws) cudaFreeAsync(s->gws, s->stream);
    cudaStreamSynchronize(s->stream);
    delete s;
}

bool angles_ok(int p, const double* x) {
    for (int k = 0; k < p; ++k)
        if (!std::isfinite(x[k])) return false;
    return true;
}

// C(z) of every z through the device's on-the-fly evaluation: uint16 cut counts (unit weights)
// or doubles (edge-weighted graphs, host_out_w).  group < 0: the default path for the size.
template <typename real>
qaoa_status cut_table_impl(const HostGraph& hg, int prec, int group, int layout, uint16_t* host_out,
                           double* host_out_w = nullptr) {
    const int n = hg.n;
    const uint64_t dim = 1ull << n;
    const size_t ob = hg.weighted ? sizeof(double) : sizeof(uint16_t);
    void* d_out = nullptr;
    CUDA_TRY(cudaMalloc(&d_out, dim * ob));
    qaoa_state_s tmp;
    tmp.n = n;
    tmp.prec = prec;
    tmp.dim = dim;
    tmp.g = hg;
    tmp.tc = tile_config_for(prec);
    tmp.stream = nullptr;
    qaoa_status st = QAOA_OK;
    if (hg.weighted) {
        const cudaError_t e = cudaMalloc(&tmp.d_wfix, wfix_bytes(hg, prec, 0));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(weight rows)");
        if (st == QAOA_OK) st = write_weight_rows<real>(&tmp);
    }
    if (st != QAOA_OK) {
    } else if (group < 0 && is_small(n, prec)) {
        SmallJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = n;
        j.synth = 1;
        j.cutval = 1;
        j.E1 = table_entries(hg);
        for (int v = 0; v < kMaxN; ++v) j.gmask[v] = v < n ? hg.upper[v] : 0;
        j.cutout = static_cast<uint16_t*>(d_out);
        j.cutout_w = static_cast<double*>(d_out);
        set_small_weights(j, hg, prec, tmp.d_wfix);
        tmp.small = true;
        tmp.dim = dim;
        st = launch_small<real>(&tmp, j);
    } else {
        constexpr int Q = PrecTraits<real>::Q;
        if (n < Q + 1) st = fail(QAOA_ERR_INVALID, "geometry cut table needs n > Q");
        if (st == QAOA_OK) {
            tmp.groups = make_groups(n, tmp.tc);
            const int grp = group < 0 ? 0 : group;
            if (grp >= (int)tmp.groups.size() || layout < 0 || layout > 2) {
                st = fail(QAOA_ERR_INVALID, "no such group or layout");
            } else {
                tmp.ntiles = 1ull << (n - Q);
                Plan plan = plan_readonly(n, tmp.tc, true, OP_CUTVAL, grp, layout);
                TileArgs<Q> a;
                std::memset(&a, 0, sizeof(a));
                fill_program<real>(a, &tmp, plan.passes[0]);
                a.cutout = static_cast<uint16_t*>(d_out);
                a.cutout_w = static_cast<double*>(d_out);
                st = launch_tile<real>(&tmp, a, 0);
            }
        }
    }
    if (st == QAOA_OK) {
        cudaError_t e = cudaMemcpy(hg.weighted ? (void*)host_out_w : (void*)host_out, d_out, dim * ob,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy(cut table)");
    }
    cudaFree(d_out);
    cudaFree(tmp.d_wfix);
    tmp.d_wfix = nullptr;
    return st;
}

}  // namespace

// ---------------------------------------------------------------------------------- allocation-free <C>
//
// qaoa_expectation_static keeps its scratch (one partial-sum pair per tile plus the final
// pair) in this file-scope device array instead of allocating workspace.  In host code
// `g_static_scratch` only names a host-side shadow, so every call looks up the array's address
// on the current device with cudaGetSymbolAddress (a table lookup inside the runtime, no
// allocation) and passes it to the kernels.  Looking it up per call, rather than caching it per
// device, keeps the address right after the device's context is torn down and rebuilt
// (cudaDeviceReset), where the array gets a new address.
namespace {

constexpr uint64_t kStaticPartials = 1ull << 16;  // tiles per call (2^16 x 16 B = 1 MiB)

}  // namespace

static __device__ __align__(256) double2 g_static_scratch[kStaticPartials + 1];

namespace {

// Graph checks of encode_graph without any heap use (repeated edges found in the bitmasks).
// A weights array is accepted when every weight is exactly 1: such a graph is the unit-weight
// graph (as for qaoa_state_init, which evaluates it with the integer cut count).
qaoa_status encode_graph_static(const qaoa_graph* g, HostGraph& hg) {
    if (!g) return fail(QAOA_ERR_INVALID, "graph is NULL");
    if (g->n < 1 || g->n > kMaxN) return fail(QAOA_ERR_INVALID, "n must be in [1, 34]");
    if (g->m < 0) return fail(QAOA_ERR_INVALID, "m must be >= 0");
    if (g->m > 0 && !g->edges) return fail(QAOA_ERR_INVALID, "edges is NULL");
    for (int e = 0; g->weights && e < g->m; ++e) {
        if (!std::isfinite(g->weights[e])) return fail(QAOA_ERR_INVALID, "non-finite edge weight");
        if (g->weights[e] != 1.0)
            return fail(QAOA_ERR_UNSUPPORTED, "edge weights other than 1 are not supported by this entry point");
    }
    hg.n = g->n;
    hg.m = g->m;
    for (int e = 0; e < g->m; ++e) {
        int u = g->edges[2 * e], v = g->edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= g->n || v >= g->n) return fail(QAOA_ERR_INVALID, "edge endpoint out of range");
        if (u == v) return fail(QAOA_ERR_INVALID, "self loop");
        if (u > v) std::swap(u, v);
        if ((hg.adj[u] >> v) & 1ull) return fail(QAOA_ERR_INVALID, "repeated edge");
        hg.upper[u] |= 1ull << v;
        hg.adj[u] |= 1ull << v;
        hg.adj[v] |= 1ull << u;
    }
    return QAOA_OK;
}

// Device address of the scratch array on the current device.
qaoa_status static_scratch(double2** out) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    *out = reinterpret_cast<double2*>(p);
    return QAOA_OK;
}

// The state must be device (or managed) memory of the current device: a host pointer, or memory
// of another device, would be read by kernels launched on the current device.  A stream that is
// being captured is refused too: the call waits for its result (cudaStreamSynchronize), which a
// capturing stream does not allow.  Neither query allocates.
qaoa_status check_static_target(const void* dev_state, cudaStream_t stream) {
    // capture first: it is the one query that is always legal while a capture is open
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(QAOA_ERR_INVALID, "the stream is being captured: this call synchronises the stream");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaPointerAttributes attr;
    std::memset(&attr, 0, sizeof(attr));
    const cudaError_t e = cudaPointerGetAttributes(&attr, dev_state);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(QAOA_ERR_INVALID, std::string("device state pointer not recognised: ") + cudaGetErrorString(e));
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(QAOA_ERR_INVALID, "device state is not device memory (host, pinned or unregistered pointer)");
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
        char msg[96];
        std::snprintf(msg, sizeof(msg), "device state lives on device %d, the current device is %d", attr.device, dev);
        return fail(QAOA_ERR_INVALID, msg);
    }
    return QAOA_OK;
}

template <typename real>
qaoa_status expectation_static_impl(const HostGraph& hg, const void* dev_state, cudaStream_t stream,
                                    double2* scratch, double* out_c, double* out_norm) {
    constexpr int Q = PrecTraits<real>::Q, R = PrecTraits<real>::R;
    using C2 = typename C2T<real>::type;
    const int n = hg.n;
    uint64_t count = 1;
    if (is_small(n, std::is_same<real, float>::value ? QAOA_C64 : QAOA_C128)) {
        SmallJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = n;
        j.E1 = hg.m + 1;
        j.expect = 1;
        j.init_amp = std::pow(2.0, -0.5 * n);
        for (int v = 0; v < kMaxN; ++v) j.gmask[v] = v < n ? hg.upper[v] : 0;
        j.state = const_cast<void*>(dev_state);
        j.partials = scratch;
        auto kfn = small_kernel<real>;
        CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
        kfn<<<1, kSmallThreads, ((size_t)1 << n) * sizeof(C2), stream>>>(j);
        CUDA_TRY(cudaGetLastError());
    } else {
        const TileConfig tc = tile_config_for(std::is_same<real, float>::value ? 0 : 1);
        count = 1ull << (n - Q);
        TileArgs<Q> a;
        std::memset(&a, 0, sizeof(a));
        fill_geometry(a, hg, low_geometry(tc), tc);
        a.nops = 2;
        a.ops[0] = Op{OP_LOAD, 0, 0, 0};
        a.ops[1] = Op{OP_EXPECT, 0, 0, 0};
        a.need_cut = 1;
        a.E1 = hg.m + 1;
        a.init_amp = std::pow(2.0, -0.5 * n);
        a.state = const_cast<void*>(dev_state);
        a.partials = scratch;
        auto kfn = tile_kernel<real, Q, R, false>;
        const size_t smem = (size_t)(1u << Q) * sizeof(C2);
        CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kfn<<<(unsigned)count, 1u << (Q - R), smem, stream>>>(a);
        CUDA_TRY(cudaGetLastError());
    }
    finalize_kernel<<<1, 1024, 0, stream>>>(scratch, count, scratch + kStaticPartials);
    CUDA_TRY(cudaGetLastError());
    double2 res;
    CUDA_TRY(cudaMemcpyAsync(&res, scratch + kStaticPartials, sizeof(double2), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (out_c) *out_c = res.x;
    if (out_norm) *out_norm = res.y;
    return QAOA_OK;
}

}  // namespace

namespace {

// Records in every RXD op of an adjoint-sweep plan how many of its level's qubits the ops before
// it (in this and earlier passes) have already turned (sweep_done): the pair terms it measures
// carry that many butterfly factors, which the complex64 sweep undoes.
void annotate_sweep(Plan& plan, int p) {
    std::vector<int> done(p, 0);
    for (Pass& ps : plan.passes)
        for (Op& op : ps.ops) {
            if (op.kind != OP_RXD) continue;
            const int level = sweep_level(op.arg);
            op.arg = (op.arg & 0x1ffff) | (done[level] << 17);
            done[level] += __builtin_popcount(op.mask);
        }
}

qaoa_status grad_workspace(qaoa_state s, int p) {
    if (p <= s->grad_levels && s->d_gtab) return QAOA_OK;
    if (s->gws) cudaFreeAsync(s->gws, s->stream);
    s->gws = nullptr;
    s->d_gtab = s->d_gmix = s->d_gwfix = nullptr;
    s->d_gacc = nullptr;
    s->d_gpart = nullptr;
    s->d_gpow = nullptr;
    s->grad_levels = 0;
    const size_t eb = elem_bytes(s->prec);
    const size_t b_tab = ws_round((size_t)p * table_entries(s->g) * eb);
    const size_t b_wfix = s->g.weighted ? ws_round(wfix_bytes(s->g, s->prec, p)) : 0;
    const size_t b_mix = ws_round((size_t)3 * p * eb);
    const size_t b_acc = ws_round(grad_acc_bytes(p));
    const size_t b_part = ws_round(grad_partials_bytes(s->n, p));
    const size_t b_pow = ws_round((size_t)p * (kMaxN + 1) * sizeof(double));
    const cudaError_t e = ws_alloc(s->dev, s->stream, b_tab + b_wfix + b_mix + b_acc + b_part + b_pow, &s->gws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->gws = nullptr;
        return fail(QAOA_ERR_OOM, std::string("gradient workspace allocation failed: ") + cudaGetErrorString(e));
    }
    char* b = static_cast<char*>(s->gws);
    s->d_gtab = b;
    b += b_tab;
    if (b_wfix) s->d_gwfix = b;
    b += b_wfix;
    s->d_gmix = b;
    b += b_mix;
    s->d_gacc = reinterpret_cast<double*>(b);
    b += b_acc;
    s->d_gpart = reinterpret_cast<double2*>(b);
    b += b_part;
    s->d_gpow = reinterpret_cast<double*>(b);
    s->grad_levels = p;
    return QAOA_OK;
}

// p forward levels from |+>^n followed by the <C> reduction into s->d_result (no host sync).
template <typename real>
qaoa_status forward_async(qaoa_state s, int p, const double* gamma, const double* beta) {
    s->lazy = true;
    s->exp_valid = false;
    s->compl_ = false;
    s->pform_ = false;
    qaoa_status st = QAOA_OK;
    for (int k0 = 0; k0 < p && st == QAOA_OK; k0 += kLayerChunk) {
        const int levels = std::min(kLayerChunk, p - k0);
        st = apply_chunk<real>(s, levels, gamma + k0, beta + k0, k0 + levels == p);
    }
    if (st != QAOA_OK) return st;
    return expectation_async<real>(s);
}

// Forward run, <C> into s->d_result and the adjoint sweep's per-level sums into s->d_gacc
// ([0, p): pair terms of d/d beta, [p, 2p): gamma terms; both without the factor 2), all
// enqueued on the state's stream without host synchronisation.  Needs grad_workspace(s, p).
template <typename real>
qaoa_status gradient_async(qaoa_state s, int p, const double* gamma, const double* beta, void* work) {
    qaoa_status st = forward_async<real>(s, p, gamma, beta);
    constexpr int Q = GradTraits<real>::Q, R = GradTraits<real>::R;
    // the tiled complex64 sweep runs in the forward passes' parity form (and folds each level's
    // butterfly factors, see rxd_parity); the one-CTA sweep and complex128 read the plain form
    const bool parity_sweep = std::is_same<real, float>::value && s->n > Q;
    if (st == QAOA_OK) st = set_parity_form<real>(s, parity_sweep);
    if (st != QAOA_OK) return st;
    using C2 = typename C2T<real>::type;
    // plain per-level tables (no folded factors) for the sweep
    for (int k0 = 0; k0 < p; k0 += kLayerChunk) {
        const int levels = std::min(kLayerChunk, p - k0);
        CoeffArgs ca;
        std::memset(&ca, 0, sizeof(ca));
        ca.levels = levels;
        ca.E1 = table_entries(s->g);
        ca.n = s->n;
        ca.fold_factors = 0;
        ca.gre = 1;
        ca.gim = 0;
        fill_coeff_weights(ca, s->g, s->prec, s->d_gwfix, 2 + k0);
        for (int k = 0; k < levels; ++k) {
            ca.gamma[k] = gamma[k0 + k];
            ca.beta[k] = beta[k0 + k];
            // packed butterflies need |t| <= 1: RX(2b) = -i X RX(2b - pi) where |tan b| > 1; X on
            // both states is an index complement, which no sweep term sees (C(~z) = C(z), and
            // X^n commutes with every X_j), and the phase (-i)^n cancels in <lambda|.|psi>
            ca.fold[k] = (parity_sweep && std::fabs(std::sin(beta[k0 + k])) > std::fabs(std::cos(beta[k0 + k]))) ? 1 : 0;
        }
        ca.sweep = parity_sweep ? 1 : 0;
        ca.gpow = s->d_gpow + (size_t)k0 * (kMaxN + 1);
        ca.phase = reinterpret_cast<C2*>(s->d_gtab) + (size_t)k0 * table_entries(s->g);
        ca.mix = reinterpret_cast<C2*>(s->d_gmix) + (size_t)3 * k0;
        dim3 grid((unsigned)std::max(1, (std::max(ca.E1, ca.m) + 255) / 256), (unsigned)levels);
        coeff_kernel<real><<<grid, 256, 0, s->stream>>>(ca);
        CUDA_TRY(cudaGetLastError());
        s->launches++;
    }
    CUDA_TRY(cudaMemsetAsync(s->d_gacc, 0, grad_acc_bytes(p), s->stream));
    if (s->n <= Q) {
        SmallGradJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = s->n;
        j.levels = p;
        j.E1 = table_entries(s->g);
        for (int v = 0; v < kMaxN; ++v) j.gmask[v] = v < s->n ? s->g.upper[v] : 0;
        j.state = s->buf;
        j.phase = s->d_gtab;
        j.mix = s->d_gmix;
        j.acc = s->d_gacc;
        set_small_weights(j, s->g, s->prec, s->d_gwfix);
        auto kfn = small_grad_kernel<real>;
        qaoa_status ast = ensure_attributes<real>();
        if (ast != QAOA_OK) return ast;
        kfn<<<1, kSmallThreadsGrad, (size_t)2 * s->dim * sizeof(C2), s->stream>>>(j);
        CUDA_TRY(cudaGetLastError());
        s->launches++;
    } else {
        Plan plan;
        const TileConfig gtc = grad_tile_config(s->prec);
        try {
            plan = plan_backward(s->n, gtc, p);
        } catch (const std::exception& ex) {
            return fail(QAOA_ERR_UNSUPPORTED, ex.what());
        }
        annotate_sweep(plan, p);
        const uint64_t gt = grad_tiles(s->n);
        const size_t smem = (size_t)2 * (1u << Q) * sizeof(C2);  // psi's and lambda's exchange tiles
        qaoa_status ast = ensure_attributes<real>();
        if (ast != QAOA_OK) return ast;
        // the passes' partials are reduced in batches of up to `chunk` passes, one launch each
        const int chunk = grad_chunk(s->n, p);
        GradBatch gb;
        gb.npass = 0;
        TileArgs<Q> a;
        for (size_t ip = 0; ip < plan.passes.size(); ++ip) {
            const Pass& ps = plan.passes[ip];
            std::memset(&a, 0, sizeof(a));
            fill_program_with(a, s, ps, plan.groups, gtc);
            a.need_cut = 1;
            a.state2 = work;
            a.phase = s->d_gtab;
            a.mix = s->d_gmix;
            a.partials = s->d_gpart + (size_t)gb.npass * 2 * gt;
            a.gpow = s->d_gpow;
            if (s->g.weighted && !fill_weighted(a, s->g, s->prec, s->d_gwfix, a.ops, a.nops))
                return fail(QAOA_ERR_UNSUPPORTED, "too many phase levels in one adjoint pass");
            int lev[2] = {-1, -1};
            for (const Op& op : ps.ops)
                if (op.kind == OP_RXD || op.kind == OP_GRADG) lev[sweep_slot(op.arg)] = sweep_level(op.arg);
            NvtxRange range("qaoa adjoint pass");
            // the persistent prefetching form where the program has one: one partial pair per CTA
            uint64_t count = gt;
            GradPfFn pf = pick_grad_pf_kernel<real>(a, s->g.weighted);
            const unsigned G = pf ? resident_ctas(pf, 1 << (Q - R), smem) : 0u;
            if (pf && G > 0) {
                count = std::min<uint64_t>(gt, G);
                pf<<<(unsigned)count, 1u << (Q - R), smem, s->stream>>>(a, gt);
            } else {
                pick_grad_kernel<real>(a, s->g.weighted)<<<(unsigned)gt, 1u << (Q - R), smem, s->stream>>>(a);
            }
            CUDA_TRY(cudaGetLastError());
            s->launches++;
            gb.lev[gb.npass][0] = lev[0];
            gb.lev[gb.npass][1] = lev[1];
            gb.cnt[gb.npass] = (uint32_t)count;
            ++gb.npass;
            if (gb.npass == chunk || ip + 1 == plan.passes.size()) {
                if (gb.npass == 1)
                    grad_reduce_kernel<<<1, 1024, 0, s->stream>>>(s->d_gpart, count, lev[0], lev[1], p, s->d_gacc);
                else
                    grad_reduce_batch_kernel<<<(unsigned)gb.npass, 1024, 0, s->stream>>>(s->d_gpart, gt, gb, p,
                                                                                       s->d_gacc);
                CUDA_TRY(cudaGetLastError());
                s->launches++;
                gb.npass = 0;
            }
        }
    }
    // the sweep consumed the state: it is |+>^n again
    s->lazy = true;
    s->exp_valid = false;
    s->compl_ = false;
    s->pform_ = false;
    return QAOA_OK;
}

template <typename real>
qaoa_status gradient_impl(qaoa_state s, int p, const double* gamma, const double* beta, void* work,
                          double* out_c, double* d_gamma, double* d_beta) {
    qaoa_status st = grad_workspace(s, p);
    if (st != QAOA_OK) return st;
    st = gradient_async<real>(s, p, gamma, beta, work);
    if (st != QAOA_OK) return st;
    std::vector<double> host(2 * (size_t)p + 2);
    CUDA_TRY(cudaMemcpyAsync(host.data(), s->d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(host.data() + 2, s->d_gacc, 2 * (size_t)p * sizeof(double), cudaMemcpyDeviceToHost,
                             s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (out_c) *out_c = host[0];
    for (int k = 0; k < p; ++k) {
        d_beta[k] = 2.0 * host[2 + k];
        d_gamma[k] = 2.0 * host[2 + p + k];
    }
    return QAOA_OK;
}

}  // namespace

extern "C" {

size_t qaoa_state_bytes(int32_t n, qaoa_prec prec) {
    if (n < 1 || n > kMaxN || (prec != QAOA_C64 && prec != QAOA_C128)) return 0;
    return (size_t)1 << n << (prec == QAOA_C64 ? 3 : 4);
}

qaoa_status qaoa_state_init(const qaoa_graph* g, qaoa_prec prec, void* dev_buf, size_t buf_bytes,
                            void* cuda_stream, qaoa_state* out) {
    if (!out) return fail(QAOA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (prec != QAOA_C64 && prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    HostGraph hg;
    qaoa_status st = encode_graph(g, hg);
    if (st != QAOA_OK) return st;
    const size_t need = qaoa_state_bytes(hg.n, prec);
    if (!dev_buf) return fail(QAOA_ERR_INVALID, "device buffer is NULL");
    if (buf_bytes < need) return fail(QAOA_ERR_INVALID, "device buffer too small");
    if (((uintptr_t)dev_buf & 15u) != 0) return fail(QAOA_ERR_INVALID, "device buffer not 16-byte aligned");

    qaoa_state s = new (std::nothrow) qaoa_state_s;
    if (!s) return fail(QAOA_ERR_OOM, "host allocation failed");
    cudaGetDevice(&s->dev);
    s->n = hg.n;
    s->prec = prec;
    s->dim = 1ull << hg.n;
    s->buf = dev_buf;
    s->stream = (cudaStream_t)cuda_stream;
    s->g = hg;
    s->tc = tile_config_for(prec);
    s->small = is_small(hg.n, prec);
    if (hg.n > s->tc.Q) {  // tiled passes (and the adjoint sweep of a small state above Q)
        s->groups = make_groups(hg.n, s->tc);
        s->ntiles = 1ull << (hg.n - s->tc.Q);
    }
    const size_t eb = elem_bytes(prec);
    const size_t b_phase = ws_round((size_t)kLayerChunk * table_entries(hg) * eb);
    const size_t b_wfix = hg.weighted ? ws_round(wfix_bytes(hg, prec, kLayerChunk)) : 0;
    const size_t b_mix = ws_round((size_t)3 * kLayerChunk * eb);
    const size_t b_part = ws_round((size_t)s->ntiles * sizeof(double2));
    const cudaError_t e = ws_alloc(s->dev, s->stream, b_phase + b_wfix + b_mix + b_part + sizeof(double2), &s->ws);
    if (e != cudaSuccess) {
        s->ws = nullptr;
        cudaGetLastError();
        release(s);
        return fail(QAOA_ERR_OOM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
    }
    char* b = static_cast<char*>(s->ws);
    s->d_phase = b;
    b += b_phase;
    if (b_wfix) s->d_wfix = b;
    b += b_wfix;
    s->d_mix = b;
    b += b_mix;
    s->d_partials = reinterpret_cast<double2*>(b);
    b += b_part;
    s->d_result = reinterpret_cast<double2*>(b);
    s->lazy = true;
    s->exp_valid = false;
    if (hg.weighted) {  // endpoint and value rows, read by <C> of a state with no level applied
        st = prec == QAOA_C64 ? write_weight_rows<float>(s) : write_weight_rows<double>(s);
        if (st != QAOA_OK) {
            release(s);
            return st;
        }
    }
    *out = s;
    return QAOA_OK;
}

qaoa_status qaoa_state_reset(qaoa_state s) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    s->lazy = true;
    s->exp_valid = false;
    s->compl_ = false;
    s->pform_ = false;
    return QAOA_OK;
}

qaoa_status qaoa_state_sync(qaoa_state s) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    CUDA_TRY(cudaSetDevice(s->dev));
    return s->prec == QAOA_C64 ? materialize<float>(s) : materialize<double>(s);
}

qaoa_status qaoa_apply_layers(qaoa_state s, int32_t p, const double* gamma, const double* beta) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    if (p < 0) return fail(QAOA_ERR_INVALID, "p must be >= 0");
    if (p > 0 && (!gamma || !beta)) return fail(QAOA_ERR_INVALID, "angle array is NULL");
    if (!angles_ok(p, gamma) || !angles_ok(p, beta)) return fail(QAOA_ERR_INVALID, "non-finite angle");
    CUDA_TRY(cudaSetDevice(s->dev));
    NvtxRange range("qaoa_apply_layers");
    if (p == 0) return s->prec == QAOA_C64 ? materialize<float>(s) : materialize<double>(s);
    for (int k0 = 0; k0 < p; k0 += kLayerChunk) {
        const int levels = std::min(kLayerChunk, p - k0);
        const bool last = (k0 + levels == p);
        qaoa_status st = s->prec == QAOA_C64 ? apply_chunk<float>(s, levels, gamma + k0, beta + k0, last)
                                             : apply_chunk<double>(s, levels, gamma + k0, beta + k0, last);
        if (st != QAOA_OK) return st;
    }
    return QAOA_OK;
}

qaoa_status qaoa_gradient(qaoa_state s, int32_t p, const double* gamma, const double* beta, void* dev_work,
                          size_t work_bytes, double* out_c, double* d_gamma, double* d_beta) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    if (p < 1) return fail(QAOA_ERR_INVALID, "p must be >= 1");
    if (!gamma || !beta || !d_gamma || !d_beta) return fail(QAOA_ERR_INVALID, "NULL array");
    if (!angles_ok(p, gamma) || !angles_ok(p, beta)) return fail(QAOA_ERR_INVALID, "non-finite angle");
    const size_t need = qaoa_state_bytes(s->n, (qaoa_prec)s->prec);
    if (!dev_work || work_bytes < need) return fail(QAOA_ERR_INVALID, "work buffer missing or too small");
    if (((uintptr_t)dev_work & 15u) != 0) return fail(QAOA_ERR_INVALID, "work buffer not 16-byte aligned");
    if (dev_work == s->buf) return fail(QAOA_ERR_INVALID, "work buffer must differ from the state buffer");
    CUDA_TRY(cudaSetDevice(s->dev));
    NvtxRange range("qaoa_gradient");
    double c = 0.0;
    qaoa_status st = s->prec == QAOA_C64 ? gradient_impl<float>(s, p, gamma, beta, dev_work, &c, d_gamma, d_beta)
                                         : gradient_impl<double>(s, p, gamma, beta, dev_work, &c, d_gamma, d_beta);
    if (st == QAOA_OK && out_c) *out_c = c;
    return st;
}

qaoa_status qaoa_expectation(qaoa_state s, double* out_c, double* out_norm) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    CUDA_TRY(cudaSetDevice(s->dev));
    return s->prec == QAOA_C64 ? expectation_impl<float>(s, out_c, out_norm)
                               : expectation_impl<double>(s, out_c, out_norm);
}

qaoa_status qaoa_state_copy_out(qaoa_state s, void* host_dst, size_t bytes) {
    if (!s || !host_dst) return fail(QAOA_ERR_INVALID, "NULL argument");
    const size_t need = qaoa_state_bytes(s->n, (qaoa_prec)s->prec);
    if (bytes < need) return fail(QAOA_ERR_INVALID, "host buffer too small");
    CUDA_TRY(cudaSetDevice(s->dev));
    qaoa_status st = s->prec == QAOA_C64 ? materialize<float>(s) : materialize<double>(s);
    if (st != QAOA_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(host_dst, s->buf, need, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QAOA_OK;
}

qaoa_status qaoa_state_free(qaoa_state s) {
    release(s);
    return QAOA_OK;
}

qaoa_status qaoa_cut_table(const qaoa_graph* g, uint16_t* host_out) {
    if (!host_out) return fail(QAOA_ERR_INVALID, "host_out is NULL");
    HostGraph hg;
    qaoa_status st = encode_graph(g, hg);
    if (st != QAOA_OK) return st;
    if (hg.weighted) return fail(QAOA_ERR_INVALID, "weighted graph: use qaoa_cut_table_f64");
    if (hg.n > 30) return fail(QAOA_ERR_INVALID, "cut table limited to n <= 30");
    return cut_table_impl<float>(hg, QAOA_C64, -1, 0, host_out);
}

qaoa_status qaoa_cut_table_f64(const qaoa_graph* g, qaoa_prec prec, int32_t group, int32_t layout, double* host_out) {
    if (!host_out) return fail(QAOA_ERR_INVALID, "host_out is NULL");
    if (prec != QAOA_C64 && prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    HostGraph hg;
    qaoa_status st = encode_graph(g, hg);
    if (st != QAOA_OK) return st;
    if (hg.n > 28) return fail(QAOA_ERR_INVALID, "cut table limited to n <= 28");
    if (!hg.weighted) {  // the cut counts, widened
        std::vector<uint16_t> c((size_t)1 << hg.n);
        st = prec == QAOA_C64 ? cut_table_impl<float>(hg, prec, group, layout, c.data())
                              : cut_table_impl<double>(hg, prec, group, layout, c.data());
        if (st == QAOA_OK)
            for (size_t z = 0; z < c.size(); ++z) host_out[z] = c[z];
        return st;
    }
    return prec == QAOA_C64 ? cut_table_impl<float>(hg, prec, group, layout, nullptr, host_out)
                            : cut_table_impl<double>(hg, prec, group, layout, nullptr, host_out);
}

qaoa_status qaoa_cut_table_geometry(const qaoa_graph* g, qaoa_prec prec, int32_t group, int32_t layout,
                                    uint16_t* host_out) {
    if (!host_out) return fail(QAOA_ERR_INVALID, "host_out is NULL");
    if (prec != QAOA_C64 && prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    if (group < 0) return fail(QAOA_ERR_INVALID, "group must be >= 0");
    HostGraph hg;
    qaoa_status st = encode_graph(g, hg);
    if (st != QAOA_OK) return st;
    if (hg.weighted) return fail(QAOA_ERR_INVALID, "weighted graph: use qaoa_cut_table_f64");
    if (hg.n > 30) return fail(QAOA_ERR_INVALID, "cut table limited to n <= 30");
    return prec == QAOA_C64 ? cut_table_impl<float>(hg, prec, group, layout, host_out)
                            : cut_table_impl<double>(hg, prec, group, layout, host_out);
}

qaoa_status qaoa_plan_describe(int32_t n, qaoa_prec prec, int32_t p, int32_t* out, int32_t cap, int32_t* count) {
    if (n < 1 || n > kMaxN || p < 0 || !count) return fail(QAOA_ERR_INVALID, "bad argument");
    if (prec != QAOA_C64 && prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    if (is_small(n, prec)) {
        *count = 0;
        return QAOA_OK;
    }
    std::vector<int32_t> d;
    try {
        Plan plan = plan_levels(n, tile_config_for(prec), p, true, true);
        d = describe(plan);
    } catch (const std::exception& ex) {
        return fail(QAOA_ERR_INVALID, ex.what());
    }
    *count = (int32_t)d.size();
    if (out)
        for (int32_t i = 0; i < std::min<int32_t>(cap, (int32_t)d.size()); ++i) out[i] = d[i];
    return QAOA_OK;
}

qaoa_status qaoa_profile_enable(qaoa_state s, int32_t enable) {
    if (!s) return fail(QAOA_ERR_INVALID, "state is NULL");
    s->prof = enable != 0;
    s->ev_used = 0;
    s->launches = 0;
    return QAOA_OK;
}

qaoa_status qaoa_debug_bounds_read(int32_t device, uint32_t* out_flags, int32_t clear) {
    if (!out_flags) return fail(QAOA_ERR_INVALID, "NULL argument");
    *out_flags = 0;
#ifdef QAOA_DEBUG_BOUNDS
    CUDA_TRY(cudaSetDevice(device));
    unsigned* p = bounds_flag_ptr();
    if (!p) return fail(QAOA_ERR_CUDA, "cannot find the index-check word on this device");
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(out_flags, p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (clear) CUDA_TRY(cudaMemset(p, 0, sizeof(unsigned)));
    return QAOA_OK;
#else
    (void)device;
    (void)clear;
    return fail(QAOA_ERR_UNSUPPORTED, "this library was built without QAOA_DEBUG_BOUNDS (index checks)");
#endif
}

qaoa_status qaoa_profile_read(qaoa_state s, qaoa_profile_stats* out) {
    if (!s || !out) return fail(QAOA_ERR_INVALID, "NULL argument");
    CUDA_TRY(cudaSetDevice(s->dev));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    std::memset(out, 0, sizeof(*out));
    out->kernel_launches = s->launches;
    const double eb = (double)elem_bytes(s->prec);
    for (size_t i = 0; i < s->ev_used; ++i) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, s->events[i].a, s->events[i].b));
        const int k = s->events[i].kind;
        if (k == 1 || k == 3 || k == 4) {
            out->pass_launches++;
            out->pass_ms += ms;
            out->pass_bytes += 2.0 * eb * (double)s->dim;
            const int c = k == 1 ? 0 : (k == 3 ? 1 : 2);
            out->kind_launches[c]++;
            out->kind_ms[c] += ms;
        } else if (k == 2) {
            out->synth_launches++;
            out->synth_ms += ms;
            out->synth_bytes += eb * (double)s->dim;
        }
    }
    return QAOA_OK;
}

qaoa_status qaoa_expectation_static(const qaoa_graph* g, qaoa_prec prec, const void* dev_state,
                                    size_t state_bytes, void* cuda_stream, double* out_c, double* out_norm) {
    if (prec != QAOA_C64 && prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    if (!dev_state) return fail(QAOA_ERR_INVALID, "device state is NULL");
    if (((uintptr_t)dev_state & 15u) != 0) return fail(QAOA_ERR_INVALID, "device state not 16-byte aligned");
    HostGraph hg;
    qaoa_status st = encode_graph_static(g, hg);
    if (st != QAOA_OK) return st;
    const int q = prec == QAOA_C64 ? PrecTraits<float>::Q : PrecTraits<double>::Q;
    if (!is_small(hg.n, prec) && (1ull << (hg.n - q)) > kStaticPartials)
        return fail(QAOA_ERR_INVALID, prec == QAOA_C64 ? "qaoa_expectation_static supports n <= 29 for complex64"
                                                       : "qaoa_expectation_static supports n <= 28 for complex128");
    if (state_bytes < qaoa_state_bytes(hg.n, prec)) return fail(QAOA_ERR_INVALID, "device state too small");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    st = check_static_target(dev_state, stream);
    if (st != QAOA_OK) return st;
    double2* scratch = nullptr;
    st = static_scratch(&scratch);
    if (st != QAOA_OK) return st;
    return prec == QAOA_C64 ? expectation_static_impl<float>(hg, dev_state, stream, scratch, out_c, out_norm)
                            : expectation_static_impl<double>(hg, dev_state, stream, scratch, out_c, out_norm);
}

const char* qaoa_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

#include "server.cuh"
