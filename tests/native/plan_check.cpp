// Host-side check of the pass planner (csrc/plan.cpp), built with AddressSanitizer and
// UndefinedBehaviorSanitizer by tests/test_host_sanitizers.py: it builds every plan the library
// can ask for (forward passes of both precisions, the adjoint sweep's tiles, read-only passes;
// n from one tile up to 34 qubits; depths 1 to 64) and checks that each is well formed.  Any
// out-of-bounds access or undefined behaviour in the planner stops the run with a report.
#include <cstdio>
#include <vector>

#include "plan.h"

using namespace qaoa;

static int g_fail = 0;
#define CHECK(cond)                                                                     \
    do {                                                                                \
        if (!(cond)) {                                                                  \
            std::fprintf(stderr, "check failed: %s (Q=%d n=%d p=%d)\n", #cond, tc.Q, n, p); \
            ++g_fail;                                                                   \
        }                                                                               \
    } while (0)

static void check_plan(const Plan& plan, const TileConfig& tc, int n, int p) {
    CHECK(!plan.passes.empty());
    for (const Pass& ps : plan.passes) {
        CHECK(ps.group >= 0 && ps.group < (int)plan.groups.size());
        CHECK(!ps.ops.empty() && (int)ps.ops.size() <= kMaxOps);
        for (const Op& op : ps.ops) {
            CHECK(op.layout <= 2);
            if (op.kind == OP_RX || op.kind == OP_RXD) CHECK(op.mask < (1u << tc.R));
        }
    }
}

int main() {
    const TileConfig configs[] = {tile_config_for(0), tile_config_for(1), TileConfig{12, 4, 3, 18}};
    const int depths[] = {1, 2, 3, 8, 64};
    int plans = 0;
    for (int c = 0; c < 3; ++c) {
        const TileConfig& tc = configs[c];
        for (int n = tc.Q + 1; n <= 34; ++n) {
            int p = 0;
            const std::vector<Group> groups = make_groups(n, tc);
            std::vector<int> seen(n, 0);
            for (const Group& g : groups) {
                CHECK(g.size() > 0 && g.size() <= tc.Q);
                for (int b : g.bits) {
                    CHECK(b >= 0 && b < n);
                    if (b >= 0 && b < n) seen[b]++;
                }
                const Geometry geo = group_geometry(g, tc);
                CHECK(geo.cprime >= 0 && geo.cprime <= tc.Q);
                (void)group_target_mask(g, tc);
            }
            for (int b = 0; b < n; ++b) CHECK(seen[b] == 1);  // the groups partition the qubits
            for (int d : depths) {
                p = d;
                if (c < 2) {
                    for (int synth = 0; synth < 2; ++synth)
                        for (int expect = 0; expect < 2; ++expect) {
                            check_plan(plan_levels(n, tc, p, synth != 0, expect != 0), tc, n, p);
                            ++plans;
                        }
                } else {
                    check_plan(plan_backward(n, tc, p), tc, n, p);
                    ++plans;
                }
            }
            p = 0;
            for (int grp = 0; grp < (int)groups.size(); ++grp)
                for (int layout = 0; layout < 3; ++layout) {
                    check_plan(plan_readonly(n, tc, false, OP_CUTVAL, grp, layout), tc, n, p);
                    ++plans;
                }
        }
    }
    std::printf("%d plans checked, %d failures\n", plans, g_fail);
    return g_fail == 0 ? 0 : 1;
}
