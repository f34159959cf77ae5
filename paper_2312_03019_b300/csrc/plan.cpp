// plan.cpp -- host-side planning of the state passes (see plan.h).
#include "plan.h"

#include <algorithm>
#include <array>
#include <climits>
#include <stdexcept>

namespace qaoa {

TileConfig tile_config_for(int prec) {
    // complex64: 2^13 amplitudes x 8 B = 64 KiB tile, 32 amplitudes per thread, 256 threads,
    //            high-group rows of >= 2^3 amplitudes (64 B); 2 MiB = 2^18 amplitudes.
    // complex128: 2^12 x 16 B = 64 KiB tile, 16 amplitudes per thread, 256 threads,
    //            high-group rows of >= 2^4 amplitudes (256 B); 2 MiB = 2^17 amplitudes.
    if (prec == 0) return TileConfig{13, 5, 3, 18};
    return TileConfig{12, 4, 4, 17};
}

// Groups for n qubits.  Group 0 holds a contiguous run [0, r) of the lowest bits (its tiles are
// rows of 2^r amplitudes) and the other groups hold at most Q - cmin bits each (their tiles keep
// >= cmin contiguous row bits).  The bits at or above the 2 MiB page boundary are dealt evenly
// over all groups, group 0 included (it gives up its top low bits for them, keeping r >= 8):
// a tile then touches 2^(its group's share) pages, and that count, not the row length, limits the
// copy rate of the scattered tiles of large states.  The remaining high groups' page bits are
// dealt round robin from the top and the mid bits (between the low run and the page boundary)
// go to the smallest group each.
std::vector<Group> make_groups(int n, const TileConfig& tc) {
    std::vector<Group> g(1);
    if (n <= tc.Q) {
        for (int b = 0; b < n; ++b) g[0].bits.push_back(b);
        return g;
    }
    const int cap = tc.Q - tc.cmin;
    const int ng = (n - tc.Q + cap - 1) / cap;  // high groups
    g.resize(1 + ng);
    const int pb = std::max(tc.page_bit, tc.Q);
    const int np = std::max(0, n - pb);  // bits [pb, n)
    const int k0 = std::min(np / (ng + 1), tc.Q - kMinLowRun);
    const int r = tc.Q - k0;
    for (int b = 0; b < r; ++b) g[0].bits.push_back(b);
    for (int b = pb; b < pb + k0; ++b) g[0].bits.push_back(b);
    int i = 0;
    for (int b = n - 1; b >= pb + k0; --b, ++i) g[1 + i % ng].bits.push_back(b);
    for (int b = r; b < std::min(pb, n); ++b) {
        int best = 1;
        for (int k = 2; k <= ng; ++k)
            if (g[k].size() < g[best].size()) best = k;
        g[best].bits.push_back(b);
    }
    for (auto& x : g) std::sort(x.bits.begin(), x.bits.end());
    return g;
}

// Tile of a group: rows of 2^c' contiguous amplitudes plus the group's remaining bits.  Group 0
// (which holds bit 0) has c' = the length of its run of low bits and applies RX to every tile
// bit; another group has c' = Q - size and applies RX to its own bits only.
Geometry group_geometry(const Group& g, const TileConfig& tc) {
    Geometry geo;
    const bool low = !g.bits.empty() && g.bits[0] == 0;
    int run = 0;
    if (low)
        while (run < g.size() && g.bits[run] == run) ++run;
    geo.cprime = low ? run : tc.Q - g.size();
    for (int u = 0; u < geo.cprime; ++u) geo.gpos[u] = u;
    for (int j = low ? run : 0, u = geo.cprime; j < g.size(); ++j, ++u) geo.gpos[u] = g.bits[j];
    return geo;
}

Geometry low_geometry(const TileConfig& tc) {
    Geometry geo;
    geo.cprime = tc.Q;
    for (int u = 0; u < tc.Q; ++u) geo.gpos[u] = u;
    return geo;
}

uint32_t group_target_mask(const Group& g, const TileConfig& tc) {
    const uint32_t all = (1u << tc.Q) - 1u;
    if (!g.bits.empty() && g.bits[0] == 0) return all;  // group 0: every tile bit
    const Geometry geo = group_geometry(g, tc);
    return all & ~((1u << geo.cprime) - 1u);
}

namespace {

// Group order of even levels; odd levels run it backwards.
std::vector<int> group_order(int g) {
    std::vector<int> order;
    if (g >= 3) {
        order.push_back(1);
        order.push_back(0);
        for (int i = 2; i < g; ++i) order.push_back(i);
    } else {
        for (int i = 0; i < g; ++i) order.push_back(i);
    }
    return order;
}

bool is_rx_like(uint8_t kind) { return kind == OP_RX || kind == OP_RXD; }

}  // namespace

Plan plan_levels(int n, const TileConfig& tc, int levels, bool synth_first, bool expect_last) {
    Plan plan;
    plan.n = n;
    plan.tc = tc;
    plan.groups = make_groups(n, tc);
    const int g = (int)plan.groups.size();
    const std::vector<int> order = group_order(g);
    for (int k = 0; k < levels; ++k) {
        for (int idx = 0; idx < g; ++idx) {
            const int grp = (k % 2 == 0) ? order[idx] : order[g - 1 - idx];
            if (idx == 0 && k > 0) {
                // same group as the last pass of level k-1: fuse phase + mixer into it
                Pass& cur = plan.passes.back();
                cur.lops.push_back(LOp{OP_PHASE, k});
                cur.lops.push_back(LOp{OP_RX, k});
                continue;
            }
            Pass ps;
            ps.group = grp;
            ps.synth = (k == 0 && idx == 0) ? synth_first : false;
            ps.store = true;
            if (idx == 0) ps.lops.push_back(LOp{OP_PHASE, k});
            ps.lops.push_back(LOp{OP_RX, k});
            plan.passes.push_back(ps);
        }
    }
    if (expect_last && !plan.passes.empty()) plan.passes.back().lops.push_back(LOp{OP_EXPECT, 0});
    assign_layouts(plan);
    return plan;
}

Plan plan_backward(int n, const TileConfig& tc, int levels) {
    Plan plan;
    plan.n = n;
    plan.tc = tc;
    plan.groups = make_groups(n, tc);
    const int g = (int)plan.groups.size();
    const std::vector<int> order = group_order(g);
    int slot = 0;  // accumulator slot of the current pass for level k
    for (int s = 0; s < levels; ++s) {
        const int k = levels - 1 - s;
        for (int idx = 0; idx < g; ++idx) {
            const int grp = (s % 2 == 0) ? order[idx] : order[g - 1 - idx];
            if (idx == 0 && s > 0) {
                slot = 1;  // second level of the fused pass
            } else {
                Pass ps;
                ps.group = grp;
                ps.synth = false;
                ps.store = true;
                if (s == 0 && idx == 0) ps.lops.push_back(LOp{OP_LAMBDA, 0});
                plan.passes.push_back(ps);
                slot = 0;
            }
            plan.passes.back().lops.push_back(LOp{OP_RXD, k | (slot << 16)});
        }
        plan.passes.back().lops.push_back(LOp{OP_GRADG, k | (slot << 16)});
        if (k > 0) plan.passes.back().lops.push_back(LOp{OP_PHASED, k});
    }
    if (!plan.passes.empty()) plan.passes.back().store = false;
    assign_layouts(plan);
    return plan;
}

Plan plan_readonly(int n, const TileConfig& tc, bool synth, uint8_t kind, int group, int layout) {
    Plan plan;
    plan.n = n;
    plan.tc = tc;
    plan.groups = make_groups(n, tc);
    Pass ps;
    ps.group = group;
    ps.synth = synth;
    ps.store = false;
    ps.lops.push_back(LOp{kind, 0});
    ps.ops.push_back(Op{(uint8_t)(synth ? OP_SYNTH : OP_LOAD), (uint8_t)layout, 0, 0});
    ps.ops.push_back(Op{kind, (uint8_t)layout, 0, 0});
    plan.passes.push_back(ps);
    return plan;
}

namespace {

struct Choice {
    int cost = INT_MAX;
    std::vector<Op> ops;
};

// All ordered sequences of distinct layouts whose register bits cover `target`, each layout
// adding at least one new bit.
std::vector<std::vector<int>> cover_sequences(const TileConfig& tc, uint32_t target) {
    std::vector<std::vector<int>> out;
    for (int subset = 1; subset < 8; ++subset) {
        std::vector<int> seq;
        for (int L = 0; L < 3; ++L)
            if ((subset >> L) & 1) seq.push_back(L);
        do {
            uint32_t covered = 0;
            bool useful = true;
            for (int L : seq) {
                const uint32_t add = tc.regMask(L) & target & ~covered;
                if (!add) useful = false;
                covered |= add;
            }
            if (useful && covered == target) out.push_back(seq);
        } while (std::next_permutation(seq.begin(), seq.end()));
    }
    return out;
}

}  // namespace

void assign_layouts(Plan& plan) {
    const TileConfig& tc = plan.tc;
    for (Pass& ps : plan.passes) {
        if (!ps.ops.empty()) continue;  // prebuilt (read-only passes)
        const uint32_t target = group_target_mask(plan.groups[ps.group], tc);
        const auto seqs = cover_sequences(tc, target);
        if (seqs.empty()) throw std::runtime_error("no layout cover for mixer group");
        // DP over the logical ops with state = current layout
        std::array<Choice, 3> st;
        for (int s = 0; s < 2; ++s) {  // programs start in a coalesced layout
            st[s].cost = 0;
            st[s].ops.push_back(Op{(uint8_t)(ps.synth ? OP_SYNTH : OP_LOAD), (uint8_t)s, 0, 0});
        }
        for (const LOp& lo : ps.lops) {
            std::array<Choice, 3> nx;
            for (int cur = 0; cur < 3; ++cur) {
                if (st[cur].cost == INT_MAX) continue;
                if (!is_rx_like(lo.kind)) {
                    Choice c = st[cur];
                    c.ops.push_back(Op{lo.kind, (uint8_t)cur, 0, lo.arg});
                    if (c.cost < nx[cur].cost) nx[cur] = c;
                    continue;
                }
                for (const auto& seq : seqs) {
                    Choice c = st[cur];
                    int L = cur;
                    uint32_t covered = 0;
                    for (int nl : seq) {
                        if (nl != L) {
                            c.ops.push_back(Op{OP_XCHG, (uint8_t)nl, 0, 0});
                            c.cost += 1;
                            L = nl;
                        }
                        const uint32_t add = tc.regMask(L) & target & ~covered;
                        covered |= add;
                        c.ops.push_back(Op{lo.kind, (uint8_t)L, (uint16_t)(add >> tc.regLo(L)), lo.arg});
                    }
                    if (c.cost < nx[L].cost) nx[L] = c;
                }
            }
            st = nx;
        }
        // finish in a coalesced layout when storing
        Choice best;
        for (int cur = 0; cur < 3; ++cur) {
            if (st[cur].cost == INT_MAX) continue;
            Choice c = st[cur];
            int L = cur;
            if (ps.store) {
                if (L == 2) {
                    c.ops.push_back(Op{OP_XCHG, 0, 0, 0});
                    c.cost += 1;
                    L = 0;
                }
                c.ops.push_back(Op{OP_STORE, (uint8_t)L, 0, 0});
            }
            if (c.cost < best.cost) best = c;
        }
        if ((int)best.ops.size() > kMaxOps) throw std::runtime_error("pass program too long");
        ps.ops = best.ops;
    }
}

std::vector<int32_t> describe(const Plan& plan) {
    std::vector<int32_t> d;
    d.push_back(plan.tc.Q);
    d.push_back(plan.tc.R);
    d.push_back(plan.tc.cmin);
    d.push_back((int32_t)plan.groups.size());
    for (const Group& g : plan.groups) {
        d.push_back(g.size());
        for (int b : g.bits) d.push_back(b);
    }
    d.push_back((int32_t)plan.passes.size());
    for (const Pass& ps : plan.passes) {
        d.push_back(ps.group);
        d.push_back((int32_t)ps.ops.size());
        for (const Op& op : ps.ops) {
            d.push_back(op.kind);
            d.push_back((op.kind == OP_RX || op.kind == OP_PHASE) ? op.arg : op.layout);
            d.push_back(op.kind == OP_RX ? (int32_t)(op.mask << plan.tc.regLo(op.layout)) : 0);
        }
    }
    return d;
}

}  // namespace qaoa
