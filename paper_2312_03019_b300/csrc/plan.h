// plan.h -- host-side planning of the state passes (no CUDA dependency).
//
// A QAOA level is a diagonal cost phase (Eq. UC_opt) followed by RX on every qubit (the mixer
// layer of Algorithm 1).  On the GPU the 2^n amplitudes are processed in tiles of 2^Q
// amplitudes held in shared memory.  A tile covers Q index bits ("local bits"): the lowest
// c' global bits (contiguous rows of 2^c' amplitudes, for coalesced HBM access) plus one
// "mixer group" of Q - c' higher global bits.  One pass streams the whole state once through
// such tiles and applies, inside each tile, the RX gates of the group's qubits; single-qubit
// RX gates on different qubits commute and the cost phase is elementwise, so a level is
// ceil-many passes over groups that together cover all n qubits.
//
// Consecutive levels reverse the group order, so the last group of level k is the first group
// of level k+1: one pass then applies RX(level k) on that group, the phase of level k+1 and
// RX(level k+1) on the same group.  A run of p levels costs p*(g-1)+1 passes instead of p*g.
// With three or more groups the order is (1, 0, 2, .., g-1): group 0, whose pass needs the most
// register-layout exchanges, is never one of the fused boundary passes.
//
// Inside a tile each thread holds 2^R amplitudes in registers.  Three register layouts
// assign R of the Q local bits to the register index (where the RX butterflies are computed
// in registers); exchanges through shared memory switch between layouts:
//   layout 0: register bits [Q-R, Q), thread bits [0, Q-R)
//   layout 1: register bits [Q-2R, Q-R), thread bits [0, Q-2R) + [Q-R, Q)
//   layout 2: register bits [0, R),      thread bits [R, Q)
// The first five thread bits are the lane bits.  Layouts 0 and 1 keep lanes on the lowest
// local bits, so global loads and stores from them are coalesced.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace qaoa {

constexpr int kMaxN = 34;
constexpr int kMaxOps = 48;
constexpr int kLayerChunk = 64;  // levels per coefficient table upload
constexpr int kMaxEdges = kMaxN * (kMaxN - 1) / 2;
constexpr int kMaxLocEdges = 13 * 12 / 2;  // edges among the Q <= 13 local bits of a tile
constexpr int kWSlots = 4;                 // weighted sums per pass: the value and up to 3 levels
constexpr int kMinLowRun = 8;              // contiguous low bits group 0 keeps (2 KiB rows complex64)

enum OpKind : uint8_t {
    OP_NONE = 0,
    OP_LOAD = 1,
    OP_SYNTH = 2,
    OP_XCHG = 3,
    OP_RX = 4,
    OP_PHASE = 5,
    OP_EXPECT = 6,
    OP_STORE = 7,
    OP_CUTVAL = 8,
    // adjoint sweep (two states: psi and lambda)
    OP_LAMBDA = 9,   // lambda <- C psi
    OP_RXD = 10,     // RX(2 beta)^dagger on both on the masked register bits, accumulating the
                     // pair terms of Im <lambda| X_j |psi> (arg = level | slot << 16)
    OP_GRADG = 11,   // accumulate sum_z C(z) Im(conj(lambda_z) psi_z) (arg = level | slot << 16)
    OP_PHASED = 12,  // exp(+i gamma_k C) on both (arg = level)
};

struct Op {
    uint8_t kind;
    uint8_t layout;  // layout after this op (LOAD/SYNTH/XCHG), or current layout
    uint16_t mask;   // RX: register-bit mask (bits of the register index)
    int32_t arg;     // RX/PHASE: level index within the chunk
};

struct TileConfig {
    int Q;         // local bits per tile
    int R;         // register bits per thread
    int cmin;      // minimum contiguous row bits in a high-group pass
    int page_bit;  // lowest index bit whose stride is >= 2 MiB (a GPU page) for this element size
    int regLo(int layout) const { return layout == 0 ? Q - R : (layout == 1 ? Q - 2 * R : 0); }
    uint32_t regMask(int layout) const { return ((1u << R) - 1u) << regLo(layout); }
    int threads() const { return 1 << (Q - R); }
};

TileConfig tile_config_for(int prec /*0 = c64, 1 = c128*/);

// A mixer group: the index bits (qubits) whose RX gates one pass applies, ascending.
struct Group {
    std::vector<int> bits;
    int size() const { return (int)bits.size(); }
};

// Tile geometry of a pass: local bits [0, cprime) are the lowest index bits (contiguous rows);
// local bit u >= cprime is index bit gpos[u].
struct Geometry {
    int cprime = 0;
    int gpos[16] = {};
};

// Logical op of a pass before layout assignment.
struct LOp {
    uint8_t kind;  // OP_PHASE, OP_RX (as a whole-group mixer), OP_EXPECT, OP_CUTVAL
    int32_t arg;   // level
};

struct Pass {
    int group;        // index into the group list
    bool synth;       // first op synthesises |+>^n instead of loading
    bool store;       // last op writes the tile back
    std::vector<LOp> lops;
    std::vector<Op> ops;  // physical program after layout assignment
};

struct Plan {
    int n = 0;
    TileConfig tc{};
    std::vector<Group> groups;
    std::vector<Pass> passes;
};

// Mixer groups for n >= Q qubits: group 0 = a run [0, r) of low bits (r >= kMinLowRun) plus its
// share of the bits at or above page_bit; the other groups hold at most Q - cmin bits each.  The
// bits at or above page_bit are spread evenly over all groups, so no tile's rows fall into more
// distinct 2 MiB pages than necessary (a tile with k group bits above page_bit touches 2^k
// pages, which measurably slows the pass down once 2^k reaches the hundreds).
std::vector<Group> make_groups(int n, const TileConfig& tc);
Geometry group_geometry(const Group& g, const TileConfig& tc);
// Geometry of the contiguous tile of bits [0, Q); allocates nothing.
Geometry low_geometry(const TileConfig& tc);
uint32_t group_target_mask(const Group& g, const TileConfig& tc);

// Passes for `levels` levels starting from a materialised state (or a deferred |+>^n when
// `synth_first`), with the expectation fused into the last pass when `expect_last`.
Plan plan_levels(int n, const TileConfig& tc, int levels, bool synth_first, bool expect_last);

// Adjoint sweep over `levels` levels (level levels-1 first) of the two states psi (state
// buffer, holding the forward result) and lambda (work buffer).  Each pass carries at most two
// levels; the level of each RXD / GRADG op and its accumulator slot are encoded in the op arg.
// The last pass stores nothing.
Plan plan_backward(int n, const TileConfig& tc, int levels);

// Single pass over one group's tiles that only evaluates (no store): expectation or cut values.
Plan plan_readonly(int n, const TileConfig& tc, bool synth, uint8_t kind, int group = 0,
                   int layout = 0);

// Assigns register layouts and shared-memory exchanges to every pass of the plan
// (minimum number of exchanges; programs start and end in layout 0 or 1).
void assign_layouts(Plan& plan);

// Flattened description (see qaoa_plan_describe in qaoa.h).
std::vector<int32_t> describe(const Plan& plan);

}  // namespace qaoa
