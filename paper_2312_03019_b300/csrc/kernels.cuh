// kernels.cuh -- sm_103a device code of the QAOA layer.
//
// Kernels:
//   coeff_kernel   per level k: phase table T_k[c] = exp(-i gamma_k c), c = 0..|E| (FP64
//                  sincos, rounded to the state precision), the mixer coefficients (cos b,
//                  sin b) and the factored butterfly t, f described at `rx`, and for
//                  edge-weighted graphs the fixed-point rows of the weighted split and the
//                  256-step rotation table of `phase_tab` in place of T_k.
//   tile_kernel    one pass over the state in tiles of 2^Q amplitudes (see plan.h): loads a
//                  tile (or synthesises |+>^n), runs the pass program (RX butterflies in
//                  registers, register-layout exchanges through swizzled shared memory, the
//                  cost phase with the on-the-fly cut count, the <C> reduction) and stores.
//                  Instantiated once interpreting any program (kNops = 0) and once per compiled
//                  pass recipe as straight-line code (kRecipe, kNops, kMasks).
//   grad_kernel    one pass of the adjoint sweep over psi and lambda = C psi (inverse mixer with
//                  the d/d beta pair sums, the d/d gamma sums, the conjugate phase), with
//   grad_reduce_kernel  the fixed-order sum of its per-tile partials per level
//                  (grad_reduce_batch_kernel: the same for a batch of passes in one launch).
//   small_kernel / small_batch_kernel / small_grad_kernel / coeff_batch_kernel
//                  a whole state of n <= Q_small qubits in shared memory, all levels in one
//                  launch: one CTA per state, many states per launch for the server.
//   finalize_kernel fixed-order FP64 sum of the per-tile partials of <C> and the norm.
//   complement_kernel resolves the pending complement and the complex64 parity form in place.
//   fill_kernel    writes |+>^n when a deferred initial state has to be materialised.
//
// On-the-fly cut count (bit-exact integer arithmetic, Algorithm 3 re-associated).  For a
// tile, split the index z into outer bits o (fixed per CTA) and the tile's local bits l.  With
// K = C(o|0), e_u = d_u^out - 2 a_u(o) (d_u^out = neighbours of local bit u outside the tile,
// a_u(o) = those set in o) and C_S the cut count of the tile-internal edges,
//     C(o|l) = K + C_S(l) + sum over set bits u of l of e_u.
// Inside a thread, l = tau | x (tau = thread bits, x = 2^R register bits), and the same split
// once more gives  C = base(tau) + sum_{j: x_j = 1} s_j(tau) + C_R(x), where C_R(x) is a
// 2^R-entry table of the register bits' internal edges.  K and e_u cost one popcount per
// vertex per CTA, base and s_j about Q + R popcounts per thread, and each amplitude two
// integer adds.
//
// Edge-weighted graphs (Algorithm 2: C(z) = sum_e w_e (z_u xor z_v) with real w_e) use the same
// split for any function F(z) = sum_e f_e (z_u xor z_v) with integer f_e, in wrapping B-bit
// arithmetic (B = 32 for complex64, 64 for complex128), so every partial sum is exact modulo
// 2^B.  Two kinds of f are used.  For the cost phase of level k, f_e = gamma_k w_e / (2 pi) in
// units of 2^-B turns, reduced modulo one turn: since z_u xor z_v is 0 or 1, the sum is
// gamma_k C(z) / (2 pi) modulo one turn up to the rounding of the m per-edge angles, and each
// amplitude turns it into exp(-i gamma_k C(z)) by one table read and a short series
// (`phase_tab`).  For <C> and the adjoint's C psi, f_e = w_e 2^S, with S
// chosen so that sum |w_e| 2^S < 2^(B-2).  Register-bit pairs enter through R(R-1)/2 pair terms
// P_jk (z_j z_k coefficients) instead of the 2^R-entry table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "plan.h"

namespace qaoa {

template <typename real>
struct C2T;
template <>
struct C2T<float> {
    using type = float2;
};
template <>
struct C2T<double> {
    using type = double2;
};

__device__ __forceinline__ float2 make_c2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 make_c2(double x, double y) { return make_double2(x, y); }

// Index checks of the debug build (-DQAOA_DEBUG_BOUNDS, `python -m paper_2312_03019_b300.build
// --debug-bounds`): a failed check sets `bit` in the word at `flag` (TileArgs::bounds_flag) and
// the access is skipped, so a wrong index is reported instead of reaching memory.  Release
// builds compile every check to `true`.  Bits: 1 state load, 2 state store, 4 shared-memory
// write, 8 shared-memory read, 16 phase-table read, 32 cut-value write, 64 weighted row read.
#ifdef QAOA_DEBUG_BOUNDS
__device__ __forceinline__ bool qaoa_in_bounds(unsigned* flag, bool ok, unsigned bit) {
    if (!ok && flag) atomicOr(flag, bit);
    return ok;
}
#define QAOA_IN_BOUNDS(flag, ok, bit) qaoa_in_bounds((flag), (ok), (bit))
#else
#define QAOA_IN_BOUNDS(flag, ok, bit) true
#endif

template <int Q>
struct TileArgs {
    int32_t n, nops, nruns;
    int32_t E1;        // entries per phase table (|E| + 1)
    int32_t need_cut;  // program evaluates C(z)
    double init_amp;   // 2^(-n/2)
    // Addressing, precomputed on the host for the pass geometry:
    uint8_t tpos[3][16];     // index bit of thread bit k (k < Q - R) in layout L
    int64_t rstep[3][8];     // element step x -> x + 1 of the register index, by ctz(x + 1)
    int64_t rstride[3][8];   // element stride of register bit j in layout L
    uint8_t run_src[kMaxN], run_len[kMaxN], run_dst[kMaxN];  // tile id bits -> outer index bits
    uint64_t gmask[kMaxN];  // graph_I rows (Table 1): bit v of gmask[u] iff edge (u, v), v > u
    uint32_t locUpper[Q];   // tile-internal upper neighbours of local bit u (local bit order)
    uint32_t locAdj[Q];     // all tile-internal neighbours of local bit u
    uint64_t outAdj[Q];     // neighbours of local bit u outside the tile (global positions)
    int32_t crtab[3][32];   // C_R(x) per register layout (32-bit words: each is an operand of
                            // the cut-index add as it is, 28.9 against 29.3 ms per fused pass
                            // at n = 33 with bytes)
    // edge-weighted graphs (pass kernels instantiated with kW)
    const void* wfix;              // rows of m fixed-point words: [0] endpoints u | v << 8,
                                   // [1] value weights, [2 + k] angles of level k
    double vscale;                 // value = (signed) sum * vscale
    int32_t m, wn, wnslots;        // edges; tile-internal edges in wloc; local slots in use
    uint32_t wloc[kMaxLocEdges];   // tile-internal edge: e | a << 10 | b << 14 (local bits a < b)
    int16_t wrow[kWSlots];         // wfix row of local slot s (slot 0: the value row)
    int8_t wslot[kLayerChunk];     // local slot holding level k's angles
    uint8_t gl2loc[kMaxN];         // local bit of index bit v, 0xff outside the tile
    double* cutout_w;              // [2^n] weighted cut values (OP_CUTVAL)
    Op ops[kMaxOps];
    void* state;
    void* state2;        // adjoint sweep: lambda
    const void* phase;   // [level][E1] complex<real>
    const void* mix;     // [3 * level + i]: (cos b, sin b), (t, 0), (f, 0) as complex<real>
    double2* partials;   // [tile] (sum |psi|^2 C, sum |psi|^2); adjoint sweep: [2 tile + slot]
    const double* gpow;  // adjoint sweep, complex64: [level][kMaxN + 1], entry s = (1 + t_level^2)^-s
    uint16_t* cutout;    // [2^n] cut values (OP_CUTVAL)
    unsigned* bounds_flag;  // debug builds: the index-check word (NULL: no reporting)
};

struct SmallJob {
    int32_t n, levels, E1;
    int32_t synth, expect, cutval, store;
    double init_amp;
    uint64_t gmask[kMaxN];
    void* state;
    const void* phase;
    const void* mix;
    double2* partials;  // one entry
    uint16_t* cutout;
    // edge-weighted graphs: wfix rows as in TileArgs (levels at rows 2 + k), NULL for unit weights
    const void* wfix;
    int32_t m;
    double vscale;
    double* cutout_w;
};

struct CoeffArgs {
    int32_t levels, E1;
    // edge-weighted graphs: also writes the fixed-point rows of wfix (endpoints and value weights
    // always, level k's angles at row wrow0 + k); E1 is then 1 (the table holds only the factor)
    int32_t weighted, m, wrow0;
    double vmul;  // 2^S of the value weights
    void* wfix;
    double w[kMaxEdges];
    uint16_t uv[kMaxEdges];  // u | v << 8
    int32_t n;                  // qubits: each level's mixer carries its factor f to the power n
    int32_t fold_factors;       // 1: multiply the phase tables by the mixers' factors (tile passes)
    int32_t fold[kLayerChunk];  // 1: the tile passes apply level k as -i X RX(2 beta - pi)
    int32_t gre, gim;           // exact factor in {1, -i, -1, i} folded into the last phase table
    // complex64 adjoint sweep: level k's table is exp(-i gamma_k c) times |f_k|^n (f_k the matched
    // factor of the level's butterflies) and gpow[k][s] = f_k^(2 s), s = 0..kMaxN
    int32_t sweep;
    double* gpow;
    double gamma[kLayerChunk];
    double beta[kLayerChunk];
    void* phase;
    void* mix;
};

constexpr int kSmallThreadsGrad = 512;

// Argument word of the adjoint sweep's RXD and GRADG ops: level in bits 0..15, accumulator slot in
// bit 16, and for RXD the number of the level's qubits whose butterflies ran before the op in
// bits 17..22 (the complex64 sweep's butterflies carry a real factor per qubit, see rxd_parity).
__host__ __device__ constexpr int sweep_level(int32_t arg) { return arg & 0xffff; }
__host__ __device__ constexpr int sweep_slot(int32_t arg) { return (arg >> 16) & 1; }
__host__ __device__ constexpr int sweep_done(int32_t arg) { return (arg >> 17) & 63; }

// ---------------------------------------------------------------------------------- helpers

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    return make_c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// d = a * b + c on two float lanes at once (one packed FMA instruction on sm_100 and later;
// CUDA's builtin, which keeps each float2 in an aligned register pair).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__host__ __device__ constexpr bool odd_parity(int x) {
    int p = 0;
    for (; x; x &= x - 1) p ^= 1;
    return p != 0;
}

// RX(2 beta) = [[c, -i s], [-i s, c]] on the pair (a, b) = (bit 0, bit 1).
template <typename C2, typename real>
__device__ __forceinline__ void rx_pair(C2& a, C2& b, real c, real s) {
    const C2 a0 = a, b0 = b;
    a = make_c2(c * a0.x + s * b0.y, c * a0.y - s * b0.x);
    b = make_c2(c * b0.x + s * a0.y, c * b0.y - s * a0.x);
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_double(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Alg. 3 cut count of z over all n vertices (graph_I rows in `gm`).
__device__ __forceinline__ int cut_count_full(const uint64_t* gm, int n, uint64_t z) {
    int c = 0;
    for (int v = 0; v < n; ++v) {
        const uint64_t bI = 0ull - ((z >> v) & 1ull);
        c += __popcll(gm[v] & (bI ^ z));
    }
    return c;
}

// ---------------------------------------------------------------------------------- weighted sums

// Fixed-point word of the weighted sums: 32 bits for complex64, 64 bits for complex128.
template <typename real>
struct WAcc;
template <>
struct WAcc<float> {
    using type = uint32_t;
    using stype = int32_t;
};
template <>
struct WAcc<double> {
    using type = uint64_t;
    using stype = int64_t;
};

// Entries per level of the weighted phase table: T[k] = g exp(-2 pi i k / kWTurnSteps), g the
// level's folded factor (T[0] = g).
constexpr int kWTurnSteps = 256;

// g exp(-2 pi i th / 2^B) from the level's table T, by angle addition (table-driven evaluation):
// the nearest step k = round(th 256 / 2^B) mod 256 comes from T, the remainder
// x = 2 pi (th - k 2^B / 256) / 2^B, |x| <= pi / 256, from the Taylor series of exp(-i x).
// complex64: cos x = 1 - x^2/2, sin x = x - x^3/6 (truncation <= x^4/24 < 1e-9, below the
// rounding of T); complex128: through x^6 and x^5 (truncation < 1e-17).
__device__ __forceinline__ float2 phase_tab(uint32_t th, const float2* __restrict__ T) {
    const int32_t r = (int32_t)(th << 8) >> 8;  // signed remainder, in [-2^23, 2^23)
    const float2 t = __ldg(T + ((th - (uint32_t)r) >> 24));
    const float x = (float)r * 1.4629180792671596e-09f;  // 2 pi / 2^32
    const float x2 = x * x;
    const float c = fmaf(-0.5f, x2, 1.0f);
    const float sn = x * fmaf(x2, -0.16666667f, 1.0f);
    return make_float2(fmaf(t.x, c, t.y * sn), fmaf(t.y, c, -t.x * sn));  // t (c - i sn)
}
__device__ __forceinline__ double2 phase_tab(uint64_t th, const double2* __restrict__ T) {
    const int64_t r = (int64_t)(th << 8) >> 8;  // signed remainder, in [-2^55, 2^55)
    const double2 t = __ldg(T + ((th - (uint64_t)r) >> 56));
    const double x = (double)r * 3.4061215800865545e-19;  // 2 pi / 2^64
    const double x2 = x * x;
    const double c = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const double sn = x * fma(x2, fma(x2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    return make_double2(fma(t.x, c, t.y * sn), fma(t.y, c, -t.x * sn));
}

template <typename WA>
__device__ __forceinline__ WA warp_sum_wrap(WA v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void smem_add(uint32_t* p, uint32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void smem_add(uint64_t* p, uint64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// F_s(z) = sum_e W[row][e] (z_u xor z_v) of one z over every edge (small states).
template <typename WA>
__device__ __forceinline__ WA wsum_full(const WA* __restrict__ W, int m, int row, uint64_t z) {
    WA acc = 0;
    const WA* f = W + (size_t)row * m;
    for (int e = 0; e < m; ++e) {
        const uint32_t uv = (uint32_t)__ldg(W + e);
        if (((z >> (uv & 255u)) ^ (z >> ((uv >> 8) & 255u))) & 1ull) acc += __ldg(f + e);
    }
    return acc;
}

// Per-CTA terms of the weighted split for every local slot s of the pass:
//   sK[s] = F_s(o|0),   sE[s][u] = sum over edges (u, v), v outside the tile, of f_e (1 - 2 o_v).
// Wrapping sums, so the result does not depend on the order of the atomics.
template <typename WA, int Q>
__device__ void weighted_cta_setup(const TileArgs<Q>& a, uint64_t zb, WA* sK, WA (*sE)[Q], uint32_t tid,
                                   uint32_t nthreads) {
    for (uint32_t i = tid; i < (uint32_t)(kWSlots * (Q + 1)); i += nthreads) {
        if (i < (uint32_t)kWSlots) sK[i] = 0;
        else sE[(i - kWSlots) / Q][(i - kWSlots) % Q] = 0;
    }
    __syncthreads();
    const WA* W = reinterpret_cast<const WA*>(a.wfix);
    WA kacc[kWSlots] = {};
    for (int e = (int)tid; e < a.m; e += (int)nthreads) {
        const uint32_t uv = (uint32_t)__ldg(W + e);
        const int u = uv & 255u, v = (uv >> 8) & 255u;
        const uint32_t bu = (uint32_t)(zb >> u) & 1u, bv = (uint32_t)(zb >> v) & 1u;
        const int lu = a.gl2loc[u], lv = a.gl2loc[v];
#pragma unroll
        for (int sl = 0; sl < kWSlots; ++sl) {
            if (sl >= a.wnslots) break;
            const WA f = __ldg(W + (size_t)a.wrow[sl] * a.m + e);
            if (bu ^ bv) kacc[sl] += f;
            if (lu != 0xff && lv == 0xff) smem_add(&sE[sl][lu], bv ? (WA)(0 - f) : f);
            if (lv != 0xff && lu == 0xff) smem_add(&sE[sl][lv], bu ? (WA)(0 - f) : f);
        }
    }
#pragma unroll
    for (int sl = 0; sl < kWSlots; ++sl) {
        const WA r = warp_sum_wrap(kacc[sl]);
        if ((tid & 31u) == 0 && sl < a.wnslots) smem_add(&sK[sl], r);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------- tile pass

template <typename real, int Q, int R, bool kGP = false, int kSw = 0>
struct Tile {
    using C2 = typename C2T<real>::type;
    static constexpr int NT = 1 << (Q - R);
    static constexpr int NE = 1 << R;
    static constexpr bool kPair = sizeof(C2) == 8;  // two amplitudes per 16-byte vector

    // complex64 amplitude forms: an amplitude is held either as (re, im) or as (im, re), such
    // that every butterfly pairs one of each and becomes two packed FMAs (see rx_bits).
    //   kGP = false (adjoint sweep): the form follows the register index, (im, re) when slot x
    //     has an odd number of set bits; it is converted wherever amplitudes leave registers.
    //   kGP = true (forward passes): the form follows the amplitude's global index z, (im, re)
    //     when z has odd parity, in registers, shared memory and HBM alike, so loads, stores and
    //     exchanges move raw values.  Slot x of a thread then holds (im, re) when
    //     parity(x) xor P = 1 with P = parity(tile outer bits) xor parity(tid) (every layout
    //     places the thread index bits by a bit permutation, so P is the same in all of them);
    //     a thread with P = 1 runs the same butterflies with t -> -t (sg = -1).  The state buffer
    //     is then in "parity form" between passes and is converted when it is read out.
    static constexpr bool kSwapOdd = kPair;
    template <int x>
    static __device__ __forceinline__ C2 to_reg(C2 z) {
        if constexpr (kSwapOdd && !kGP && odd_parity(x)) return make_c2(z.y, z.x);
        else return z;
    }
    template <int x>
    static __device__ __forceinline__ C2 from_reg(C2 z) { return to_reg<x>(z); }
    // real / imaginary part of the amplitude in slot x, and a slot value from (re, im)
    template <int x>
    static __device__ __forceinline__ real re_of(C2 z) {
        if constexpr (kSwapOdd && odd_parity(x)) return z.y;
        else return z.x;
    }
    template <int x>
    static __device__ __forceinline__ real im_of(C2 z) {
        if constexpr (kSwapOdd && odd_parity(x)) return z.x;
        else return z.y;
    }
    template <int x>
    static __device__ __forceinline__ C2 mk(real re, real im) { return to_reg<x>(make_c2(re, im)); }

    static __host__ __device__ constexpr int rlo(int L) { return L == 0 ? Q - R : (L == 1 ? Q - 2 * R : 0); }

    // Shared-memory index swizzle.  It is linear over GF(2) (phys(a ^ b) = phys(a) ^ phys(b)), so
    // an element's address is a per-thread constant XOR a compile-time constant.
    //   complex64 (8 B, Q = 13): bits 1..3 ^= (l5, l6, l7 ^ l8).  Bit 0 is kept, so each pair
    //     (l, l ^ 1) stays one aligned 16-byte vector.  8-byte accesses of layouts 0 and 1 hit 16
    //     distinct 8-byte slots per half warp; layout 2 moves pairs with 16-byte accesses, 8
    //     distinct 16-byte slots per quarter warp.
    //   complex64 passes that use layouts 0 and 1 only (kSw = 1): bit 3 ^= l8, which is enough
    //     for those two (a half warp covers l0..l3 in layout 0, where l8 is a register bit, and
    //     l0..l2, l8 in layout 1, where l3 is one), and leaves the register bits of both layouts
    //     apart from the thread bits but for bit 3: an address is one of two per-thread bases
    //     plus a compile-time offset (see to_smem).
    //   complex128 (16 B, Q = 12): bits 0..4 ^= bits 4..8; 8 distinct slots per quarter warp in
    //     every layout.
    static __host__ __device__ constexpr uint32_t swz(uint32_t l) {
        if (kPair && kSw == 1) return l ^ (((l >> 8) & 1u) << 3);
        return kPair ? (l ^ (((l >> 4) & 14u) ^ ((l >> 5) & 8u))) : (l ^ ((l >> 4) & 31u));
    }
    // kSw = 1, layouts 0 and 1: the byte offset of register slot x is P_b + off(x), P_b the
    // thread's swizzled base with bit 3 flipped by b = x & 1 (l8 in layout 0, l3 in layout 1),
    // off(x) the rest of x's bits (l9..l12 / l4..l7), disjoint from every thread bit.
    template <int L, int x>
    static __host__ __device__ constexpr uint32_t sw1_off() {
        return L == 0 ? ((uint32_t)x << 8) * 8u : ((uint32_t)(x >> 1) << 4) * 8u;
    }

    // local bits of thread `tid` in layout L (register bits zero)
    static __device__ __forceinline__ uint32_t tbits(int L, uint32_t tid) {
        if (L == 0) return tid;
        if (L == 1) {
            constexpr int lo = Q - 2 * R;
            return (tid & ((1u << lo) - 1u)) | ((tid >> lo) << (Q - R));
        }
        return tid << R;
    }

    struct Ctx {
        uint64_t zb;  // outer bits of the tile
        int K;
        const TileArgs<Q>* a;
        int* sE;
        const void* wK;  // weighted: per-slot F_s(o|0) (shared memory)
        const void* wE;  // weighted: per-slot e_u terms, [slot][Q] (shared memory)
        real sg;         // kGP: +1, or -1 when the thread's even-parity slots hold (im, re)
    };

    // f applied to the amplitude in slot x: f itself on a (re, im) slot, conj(f) on an (im, re)
    // slot (the complex product of the raw pair with conj(f) is the swapped product).
    template <int x>
    static __device__ __forceinline__ C2 apply_phase(C2 vx, C2 f, real sg) {
        if constexpr (kSwapOdd && kGP) {
            const real fy = (odd_parity(x) ? -sg : sg) * f.y;
            return cmul(vx, make_c2(f.x, fy));
        } else if constexpr (kSwapOdd && odd_parity(x)) {
            return make_c2(vx.x * f.x + vx.y * f.y, vx.y * f.x - vx.x * f.y);
        } else {
            return cmul(vx, f);
        }
    }

    using WA = typename WAcc<real>::type;
    using SWA = typename WAcc<real>::stype;
    static constexpr int NP = R * (R - 1) / 2;

    template <int N>
    static __device__ __forceinline__ void add_at(WA (&s)[N], int idx, WA v) {
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j == idx) s[j] += v;
    }
    static __device__ __forceinline__ void add_pair(WA (&P)[NP], int ja, int jb, WA v) {
        int q = 0;
#pragma unroll
        for (int j = 0; j < R; ++j)
#pragma unroll
            for (int k = j + 1; k < R; ++k) {
                if (j == ja && k == jb) P[q] += v;
                ++q;
            }
    }

    // Weighted split of local slot ls in layout L: F = base(tau) + sum_{j in x} s_j
    // + sum_{j < k in x} P_jk.  The tile-internal edges are classified by where their ends sit:
    // two thread bits (into base), a register and a thread bit (a slope), two register bits (two
    // slopes and a pair term).
    template <int L>
    static __device__ __forceinline__ WA wsetup(const Ctx& c, uint32_t tid, int ls, WA (&s)[R], WA (&P)[NP]) {
        const TileArgs<Q>& a = *c.a;
        const uint32_t tau = tbits(L, tid);
        const WA* sE = reinterpret_cast<const WA*>(c.wE) + ls * Q;
        WA base = reinterpret_cast<const WA*>(c.wK)[ls];
#pragma unroll
        for (int u = 0; u < Q; ++u)
            if ((tau >> u) & 1u) base += sE[u];
#pragma unroll
        for (int j = 0; j < R; ++j) s[j] = sE[rlo(L) + j];
#pragma unroll
        for (int q = 0; q < NP; ++q) P[q] = 0;
        const WA* __restrict__ W = reinterpret_cast<const WA*>(a.wfix) + (size_t)a.wrow[ls] * a.m;
        for (int i = 0; i < a.wn; ++i) {
            const uint32_t ent = a.wloc[i];
            const WA f = QAOA_IN_BOUNDS(a.bounds_flag, (int)(ent & 1023u) < a.m, 64u) ? __ldg(W + (ent & 1023u)) : (WA)0;
            const int ua = (ent >> 10) & 15, ub = (ent >> 14) & 15;
            const int ja = ua - rlo(L), jb = ub - rlo(L);
            const bool ra = (unsigned)ja < (unsigned)R, rb = (unsigned)jb < (unsigned)R;
            const uint32_t ta = (tau >> ua) & 1u, tb = (tau >> ub) & 1u;
            if (ra && rb) {
                add_at(s, ja, f);
                add_at(s, jb, f);
                add_pair(P, ja, jb, (WA)(0 - 2 * f));
            } else if (ra) {
                if (tb) base += f;
                add_at(s, ja, tb ? (WA)(0 - f) : f);
            } else if (rb) {
                if (ta) base += f;
                add_at(s, jb, ta ? (WA)(0 - f) : f);
            } else if (ta ^ tb) {
                base += f;
            }
        }
        return base;
    }

    template <int x>
    static __device__ __forceinline__ WA wat(WA base, const WA (&s)[R], const WA (&P)[NP]) {
        WA v = base;
#pragma unroll
        for (int j = 0; j < R; ++j)
            if ((x >> j) & 1) v += s[j];
        int q = 0;
#pragma unroll
        for (int j = 0; j < R; ++j)
#pragma unroll
            for (int k = j + 1; k < R; ++k) {
                if (((x >> j) & 1) && ((x >> k) & 1)) v += P[q];
                ++q;
            }
        return v;
    }

    static __device__ __forceinline__ real wval(WA v, double scale) { return (real)((double)(SWA)v * scale); }

    // Element offset of the thread's register-index-0 amplitude in layout L (thread bits only).
    template <int L>
    static __device__ __forceinline__ uint64_t toff(const TileArgs<Q>& a, uint32_t tid) {
        uint64_t o = 0;
#pragma unroll
        for (int k = 0; k < Q - R; ++k)
            if ((tid >> k) & 1u) o |= 1ull << a.tpos[L][k];
        return o;
    }

    // Calls f(std::integral_constant<int, x>) for x = 0 .. N-1 (compile-time register indices).
    template <int N, typename F, int x = 0>
    static __device__ __forceinline__ void for_x(F&& f) {
        if constexpr (x < N) {
            f(std::integral_constant<int, x>{});
            for_x<N, F, x + 1>(static_cast<F&&>(f));
        }
    }

    static __host__ __device__ constexpr int ctz_next(int x) {
        int j = 0;
        while ((((x + 1) >> j) & 1) == 0) ++j;
        return j;
    }

    template <int L>
    static __device__ __forceinline__ void load(C2 (&v)[NE], const Ctx& c, uint32_t tid) {
        load_from<L>(v, c, tid, c.a->state);
    }

    template <int L>
    static __device__ __forceinline__ void store(const C2 (&v)[NE], const Ctx& c, uint32_t tid) {
        store_to<L>(v, c, tid, c.a->state);
    }

    template <int L>
    static __device__ __forceinline__ void load_from(C2 (&v)[NE], const Ctx& c, uint32_t tid, const void* base) {
        const TileArgs<Q>& a = *c.a;
        const C2* g = reinterpret_cast<const C2*>(base) + c.zb + toff<L>(a, tid);
        int64_t d[R];
#pragma unroll
        for (int j = 0; j < R; ++j) d[j] = a.rstep[L][j];
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            if (QAOA_IN_BOUNDS(a.bounds_flag, (uint64_t)(g - reinterpret_cast<const C2*>(base)) >> a.n == 0, 1u))
                v[x] = to_reg<x>(*g);
            else
                v[x] = make_c2((real)0, (real)0);
            if constexpr (x + 1 < NE) g += d[ctz_next(x)];
        });
    }

    template <int L>
    static __device__ __forceinline__ void store_to(const C2 (&v)[NE], const Ctx& c, uint32_t tid, void* base) {
        const TileArgs<Q>& a = *c.a;
        C2* g = reinterpret_cast<C2*>(base) + c.zb + toff<L>(a, tid);
        int64_t d[R];
#pragma unroll
        for (int j = 0; j < R; ++j) d[j] = a.rstep[L][j];
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            if (QAOA_IN_BOUNDS(a.bounds_flag, (uint64_t)(g - reinterpret_cast<C2*>(base)) >> a.n == 0, 2u))
                *g = from_reg<x>(v[x]);
            if constexpr (x + 1 < NE) g += d[ctz_next(x)];
        });
    }

    // Shared-memory exchange: byte offset = (swizzled thread part) XOR (compile-time register part).
    // An exchange from layout Lp writes each of the thread's amplitudes at the position its index
    // maps to, which is exactly where the thread read them in the previous exchange (whose target
    // layout was Lp); so one barrier, between the writes and the reads, is enough: no thread can
    // overwrite a position another thread has still to read.  A pass's first exchange finds the
    // tile unused (one tile per CTA).
    template <int L>
    static __device__ __forceinline__ void to_smem(const C2 (&v)[NE], unsigned char* tile, uint32_t tid,
                                                   unsigned* bf = nullptr) {
        constexpr uint32_t kBytes = (1u << Q) * (uint32_t)sizeof(C2);
        const uint32_t P = swz(tbits(L, tid)) * (uint32_t)sizeof(C2);
        if constexpr (kPair && kSw == 1 && L != 2) {
            const uint32_t Pb[2] = {P, P ^ 64u};
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const uint32_t o = Pb[x & 1] + sw1_off<L, x>();
                if (QAOA_IN_BOUNDS(bf, o + 8u <= kBytes, 4u)) *reinterpret_cast<C2*>(tile + o) = from_reg<x>(v[x]);
            });
        } else if constexpr (kPair && L == 2) {  // register bit 0 is local bit 0: store amplitude pairs
            for_x<NE / 2>([&](auto H) {
                constexpr int x = 2 * decltype(H)::value;
                const C2 a = from_reg<x>(v[x]), b = from_reg<x + 1>(v[x + 1]);
                const uint32_t o = P ^ (swz((uint32_t)x) * 8u);
                if (QAOA_IN_BOUNDS(bf, o + 16u <= kBytes && (o & 15u) == 0, 4u))
                    *reinterpret_cast<float4*>(tile + o) = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
            });
        } else {
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const uint32_t o = P ^ (swz((uint32_t)x << rlo(L)) * (uint32_t)sizeof(C2));
                if (QAOA_IN_BOUNDS(bf, o + (uint32_t)sizeof(C2) <= kBytes, 4u))
                    *reinterpret_cast<C2*>(tile + o) = from_reg<x>(v[x]);
            });
        }
    }

    template <int L>
    static __device__ __forceinline__ void from_smem(C2 (&v)[NE], const unsigned char* tile, uint32_t tid,
                                                     unsigned* bf = nullptr) {
        constexpr uint32_t kBytes = (1u << Q) * (uint32_t)sizeof(C2);
        const uint32_t P = swz(tbits(L, tid)) * (uint32_t)sizeof(C2);
        if constexpr (kPair && kSw == 1 && L != 2) {
            const uint32_t Pb[2] = {P, P ^ 64u};
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const uint32_t o = Pb[x & 1] + sw1_off<L, x>();
                if (QAOA_IN_BOUNDS(bf, o + 8u <= kBytes, 8u))
                    v[x] = to_reg<x>(*reinterpret_cast<const C2*>(tile + o));
                else
                    v[x] = make_c2((real)0, (real)0);
            });
        } else if constexpr (kPair && L == 2) {
            for_x<NE / 2>([&](auto H) {
                constexpr int x = 2 * decltype(H)::value;
                const uint32_t o = P ^ (swz((uint32_t)x) * 8u);
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (QAOA_IN_BOUNDS(bf, o + 16u <= kBytes && (o & 15u) == 0, 8u))
                    q = *reinterpret_cast<const float4*>(tile + o);
                v[x] = to_reg<x>(make_c2((real)q.x, (real)q.y));
                v[x + 1] = to_reg<x + 1>(make_c2((real)q.z, (real)q.w));
            });
        } else {
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const uint32_t o = P ^ (swz((uint32_t)x << rlo(L)) * (uint32_t)sizeof(C2));
                if (QAOA_IN_BOUNDS(bf, o + (uint32_t)sizeof(C2) <= kBytes, 8u))
                    v[x] = to_reg<x>(*reinterpret_cast<const C2*>(tile + o));
                else
                    v[x] = make_c2((real)0, (real)0);
            });
        }
    }

    // Issues one 8-byte cp.async per amplitude of the thread in layout L (the elements load_from
    // reads) into that element's place in a shared-memory tile (where from_smem, in any layout,
    // reads it).  The values are copied raw, so this serves the forms that keep amplitudes as
    // stored (kGP).  Completed by cp.async.wait_all in the caller, then a CTA barrier.
    template <int L>
    static __device__ __forceinline__ void prefetch_to(unsigned char* tile, const Ctx& c, uint32_t tid,
                                                       const void* base, unsigned* bf = nullptr) {
        static_assert(kPair && kGP && kSw == 0, "raw 8-byte copies in the default swizzle");
        constexpr uint32_t kBytes = (1u << Q) * (uint32_t)sizeof(C2);
        const TileArgs<Q>& a = *c.a;
        const C2* g = reinterpret_cast<const C2*>(base) + c.zb + toff<L>(a, tid);
        int64_t d[R];
#pragma unroll
        for (int j = 0; j < R; ++j) d[j] = a.rstep[L][j];
        const uint32_t P = swz(tbits(L, tid)) * (uint32_t)sizeof(C2);
        const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(tile);
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            const uint32_t o = P ^ (swz((uint32_t)x << rlo(L)) * (uint32_t)sizeof(C2));
            if (QAOA_IN_BOUNDS(bf, ((uint64_t)(g - reinterpret_cast<const C2*>(base)) >> a.n) == 0 && o + 8u <= kBytes,
                               1u))
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s0 + o), "l"(g) : "memory");
            if constexpr (x + 1 < NE) g += d[ctz_next(x)];
        });
    }

    // base(tau) and slopes s_j of the on-the-fly cut count in layout L
    template <int L>
    static __device__ __forceinline__ int cut_setup(const Ctx& c, uint32_t tid, int (&s)[R]) {
        const TileArgs<Q>& a = *c.a;
        const uint32_t tau = tbits(L, tid);
        int cs = 0, e = 0;
#pragma unroll
        for (int u = 0; u < Q; ++u) {
            const uint32_t bit = (tau >> u) & 1u;
            cs += __popc(a.locUpper[u] & (tau ^ (0u - bit)));
            e += bit ? c.sE[u] : 0;
        }
        constexpr uint32_t RM = ((1u << R) - 1u) << rlo(L);
        constexpr uint32_t TM = ((1u << Q) - 1u) & ~RM;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int u = rlo(L) + j;
            s[j] = c.sE[u] + __popc(a.locAdj[u] & TM) - 2 * __popc(a.locAdj[u] & tau);
        }
        return c.K + cs + e;
    }

    template <int x>
    static __device__ __forceinline__ int cut_at(int base, const int (&s)[R], const uint8_t* cr) {
        int cidx = base + cr[x];
#pragma unroll
        for (int j = 0; j < R; ++j)
            if ((x >> j) & 1) cidx += s[j];
        return cidx;
    }

    template <int L, bool kW = false>
    static __device__ __forceinline__ void phase(C2 (&v)[NE], const Ctx& c, uint32_t tid, int level) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {  // the level's table holds kWTurnSteps rotations of the folded factor
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, a.wslot[level], s, P);
            const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                v[x] = apply_phase<x>(v[x], phase_tab(wat<x>(base, s, P), T), c.sg);
            });
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            // the count is exact and always in [0, |E|] (the debug build checks every read)
            (void)QAOA_IN_BOUNDS(a.bounds_flag, (unsigned)cidx < (unsigned)a.E1, 16u);
            v[x] = apply_phase<x>(v[x], __ldg(T + cidx), c.sg);
        });
    }

    template <int L, bool kW = false>
    static __device__ __forceinline__ void expect(const C2 (&v)[NE], const Ctx& c, uint32_t tid,
                                                  double& accC, double& accN) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, 0, s, P);
            real sc = 0, sn = 0;  // sc in the value rows' fixed-point unit, scaled once below
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const real p = v[x].x * v[x].x + v[x].y * v[x].y;
                sn += p;
                sc += p * (real)(SWA)wat<x>(base, s, P);
            });
            accC += (double)sc * a.vscale;
            accN += (double)sn;
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        real sc = 0, sn = 0;
#pragma unroll
        for (int x = 0; x < NE; ++x) {
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            const real p = v[x].x * v[x].x + v[x].y * v[x].y;
            sn += p;
            sc += p * (real)cidx;
        }
        accC += (double)sc;
        accN += (double)sn;
    }

    template <int L, bool kW = false>
    static __device__ __forceinline__ void cutval(const Ctx& c, uint32_t tid) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, 0, s, P);
            double* __restrict__ g = a.cutout_w + c.zb + toff<L>(a, tid);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                int64_t o = 0;
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if ((x >> j) & 1) o += a.rstride[L][j];
                if (QAOA_IN_BOUNDS(a.bounds_flag, (uint64_t)(g + o - a.cutout_w) >> a.n == 0, 32u))
                    g[o] = (double)(SWA)wat<x>(base, s, P) * a.vscale;
            });
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        uint16_t* __restrict__ g = a.cutout + c.zb + toff<L>(a, tid);
#pragma unroll
        for (int x = 0; x < NE; ++x) {
            int cidx = base + a.crtab[L][x];
            int64_t o = 0;
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) {
                    cidx += s[j];
                    o += a.rstride[L][j];
                }
            if (QAOA_IN_BOUNDS(a.bounds_flag, (uint64_t)(g + o - a.cutout) >> a.n == 0, 32u)) g[o] = (uint16_t)cidx;
        }
    }

    // ------------------------------------------------------------ adjoint sweep (psi v, lambda w)

    // lambda <- C psi
    template <int L, bool kW = false>
    static __device__ __forceinline__ void lambda_init(const C2 (&v)[NE], C2 (&w)[NE], const Ctx& c, uint32_t tid) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, 0, s, P);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const real cc = wval(wat<x>(base, s, P), a.vscale);
                w[x] = make_c2(cc * v[x].x, cc * v[x].y);
            });
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            const real cc = (real)cidx;
            w[x] = make_c2(cc * v[x].x, cc * v[x].y);
        });
    }

    // RX(2b)^dagger = [[c, is], [is, c]] on both states for the masked register bits; before each
    // butterfly adds Im(conj(l_a) p_b + conj(l_b) p_a), the pair terms of Im <lambda| X_j |psi>.
    static __device__ __forceinline__ real rx_dual(C2 (&v)[NE], C2 (&w)[NE], uint32_t mask, real cb, real sb) {
        real acc = 0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (!((mask >> j) & 1u)) continue;
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                if (!(x & (1 << j))) {
                    const int y = x | (1 << j);
                    const real ar = re_of<x>(v[x]), ai = im_of<x>(v[x]);
                    // y differs from x in one bit: its slot form is the opposite one
                    const real br = (kSwapOdd && !odd_parity(x)) ? v[y].y : v[y].x;
                    const real bi = (kSwapOdd && !odd_parity(x)) ? v[y].x : v[y].y;
                    const real lar = re_of<x>(w[x]), lai = im_of<x>(w[x]);
                    const real lbr = (kSwapOdd && !odd_parity(x)) ? w[y].y : w[y].x;
                    const real lbi = (kSwapOdd && !odd_parity(x)) ? w[y].x : w[y].y;
                    acc += (lar * bi - lai * br) + (lbr * ai - lbi * ar);
                    const real nar = cb * ar - sb * bi, nai = cb * ai + sb * br;
                    const real nbr = cb * br - sb * ai, nbi = cb * bi + sb * ar;
                    const real nlar = cb * lar - sb * lbi, nlai = cb * lai + sb * lbr;
                    const real nlbr = cb * lbr - sb * lai, nlbi = cb * lbi + sb * lar;
                    v[x] = mk<x>(nar, nai);
                    w[x] = mk<x>(nlar, nlai);
                    if (kSwapOdd && !odd_parity(x)) {
                        v[y] = make_c2(nbi, nbr);
                        w[y] = make_c2(nlbi, nlbr);
                    } else {
                        v[y] = make_c2(nbr, nbi);
                        w[y] = make_c2(nlbr, nlbi);
                    }
                }
            });
        }
        return acc;
    }

    // complex64 adjoint sweep in the parity form (kGP): RX(2 beta)^dagger on psi (v) and lambda
    // (w) for the masked register bits as the butterflies a' = a + i t b, b' = b + i t a (one
    // packed FMA per amplitude per state; `tn` = -sg t), which leave a real factor 1/f with
    // f^2 = 1 / (1 + t^2) on every amplitude of both states per qubit.  Before the butterflies it
    // sums the pair terms Im(conj(l_a) p_b + conj(l_b) p_a) of Im <lambda| X_j |psi> over the masked
    // bits j: a pair term of level k is unchanged by the level's RX gates on either state (they
    // commute with X_j), so measured before this op's butterflies it is the true term times
    // (1/f^2)^s, s = the level's qubits done before the op; the caller applies f^(2 s).  With x
    // the even-parity slot of a pair (the (re, im) form when P = 0) and y the other, the term is
    // (E.x - E.y) - (F.x - F.y) with E = w[x] v[y] and F = w[y] v[x] componentwise; a thread with
    // P = 1 has every form flipped and gets the negative, so the caller also multiplies by sg.
    // kFixed: 0 for a runtime mask, else 32 | the register mask compiled in (no per-bit branches)
    template <bool kScalar = false, uint32_t kFixed = 0>
    static __device__ __forceinline__ real rxd_parity(C2 (&v)[NE], C2 (&w)[NE], uint32_t mask, real tn) {
        auto on = [&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr ((kFixed & 32u) != 0) return ((kFixed >> j) & 1u) != 0;
            else return ((mask >> j) & 1u) != 0;
        };
        // d += a * b componentwise, packed (FFMA2) or as two FMAs (bit-identical)
        auto acc2 = [](C2 a, C2 b, C2 d) -> C2 {
            if constexpr (kScalar) return make_c2(fma(a.x, b.x, d.x), fma(a.y, b.y, d.y));
            else return ffma2(a, b, d);
        };
        C2 E0 = make_c2((real)0, (real)0), F0 = E0, E1 = E0, F1 = E0;
        for_x<R>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if (!on(J)) return;
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                if constexpr (!(x & (1 << j))) {
                    constexpr int y = x | (1 << j);
                    constexpr int xe = odd_parity(x) ? y : x, xo = odd_parity(x) ? x : y;
                    if constexpr (j % 2 == 0) {
                        E0 = acc2(w[xe], v[xo], E0);
                        F0 = acc2(w[xo], v[xe], F0);
                    } else {
                        E1 = acc2(w[xe], v[xo], E1);
                        F1 = acc2(w[xo], v[xe], F1);
                    }
                }
            });
        });
        for_x<R>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if (!on(J)) return;
            const C2 cp = make_c2(tn, -tn), cm = make_c2(-tn, tn);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                if constexpr (!(x & (1 << j))) {
                    constexpr int y = x | (1 << j);
                    constexpr int xn = odd_parity(x) ? y : x, xs = odd_parity(x) ? x : y;
                    bfly<kScalar>(v[xn], v[xs], cp, cm);
                    bfly<kScalar>(w[xn], w[xs], cp, cm);
                }
            });
        });
        return ((E0.x - E0.y) - (F0.x - F0.y)) + ((E1.x - E1.y) - (F1.x - F1.y));
    }

    // complex64 sweep (kGP): sum_z C(z) Im(conj(lambda_z) psi_z) for the P = 0 orientation (the
    // caller multiplies by sg): a (re, im) slot gives w.x v.y - w.y v.x, an (im, re) slot its
    // negative.
    template <int L, bool kW = false>
    static __device__ __forceinline__ real grad_gamma_parity(const C2 (&v)[NE], const C2 (&w)[NE], const Ctx& c,
                                                             uint32_t tid) {
        const TileArgs<Q>& a = *c.a;
        real acc_e = 0, acc_o = 0;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, 0, s, P);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const real d = (real)(SWA)wat<x>(base, s, P) * (w[x].x * v[x].y - w[x].y * v[x].x);
                if constexpr (odd_parity(x)) acc_o += d;
                else acc_e += d;
            });
            return (real)((double)(acc_e - acc_o) * a.vscale);
        } else {
            int s[R];
            const int base = cut_setup<L>(c, tid, s);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                int cidx = base + a.crtab[L][x];
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if ((x >> j) & 1) cidx += s[j];
                const real d = (real)cidx * (w[x].x * v[x].y - w[x].y * v[x].x);
                if constexpr (odd_parity(x)) acc_o += d;
                else acc_e += d;
            });
            return acc_e - acc_o;
        }
    }

    // complex64 sweep (kGP): exp(+i gamma C(z)) times the table's real factor on both states: the
    // conjugate of the table entry applied in the slot's form (as in `phase`).
    template <int L, bool kW = false>
    static __device__ __forceinline__ void phase_dual_parity(C2 (&v)[NE], C2 (&w)[NE], const Ctx& c, uint32_t tid,
                                                             int level) {
        const TileArgs<Q>& a = *c.a;
        const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, a.wslot[level], s, P);
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const C2 f = phase_tab(wat<x>(base, s, P), T);
                const C2 fc = make_c2(f.x, -f.y);
                v[x] = apply_phase<x>(v[x], fc, c.sg);
                w[x] = apply_phase<x>(w[x], fc, c.sg);
            });
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            (void)QAOA_IN_BOUNDS(a.bounds_flag, (unsigned)cidx < (unsigned)a.E1, 16u);
            const C2 f = __ldg(T + min((unsigned)cidx, (unsigned)(a.E1 - 1)));
            const C2 fc = make_c2(f.x, -f.y);
            v[x] = apply_phase<x>(v[x], fc, c.sg);
            w[x] = apply_phase<x>(w[x], fc, c.sg);
        });
    }

    // grad_gamma_parity followed by phase_dual_parity in the same layout (unit weights), with
    // each amplitude's cut value counted once for both: the gamma term of slot x is taken from
    // the amplitudes before their phase, the sums run in the same order, so the results are
    // bit-identical to the two ops in turn.  The cut value is exact, so the table index needs no
    // clamp (the debug build checks it).
    template <int L>
    static __device__ __forceinline__ real grad_gamma_phase_dual_parity(C2 (&v)[NE], C2 (&w)[NE], const Ctx& c,
                                                                        uint32_t tid, int level) {
        const TileArgs<Q>& a = *c.a;
        const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
        real acc_e = 0, acc_o = 0;
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            const real d = (real)cidx * (w[x].x * v[x].y - w[x].y * v[x].x);
            if constexpr (odd_parity(x)) acc_o += d;
            else acc_e += d;
            (void)QAOA_IN_BOUNDS(a.bounds_flag, (unsigned)cidx < (unsigned)a.E1, 16u);
            const C2 f = __ldg(T + cidx);
            const C2 fc = make_c2(f.x, -f.y);
            v[x] = apply_phase<x>(v[x], fc, c.sg);
            w[x] = apply_phase<x>(w[x], fc, c.sg);
        });
        return acc_e - acc_o;
    }

    // sum_z C(z) Im(conj(lambda_z) psi_z) over the thread's amplitudes
    template <int L, bool kW = false>
    static __device__ __forceinline__ real grad_gamma(const C2 (&v)[NE], const C2 (&w)[NE], const Ctx& c, uint32_t tid) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, 0, s, P);
            real acc = 0;  // in the value rows' fixed-point unit, scaled once at the end
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                acc += (real)(SWA)wat<x>(base, s, P) *
                       (re_of<x>(w[x]) * im_of<x>(v[x]) - im_of<x>(w[x]) * re_of<x>(v[x]));
            });
            return (real)((double)acc * a.vscale);
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        real acc = 0;
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            acc += (real)cidx * (re_of<x>(w[x]) * im_of<x>(v[x]) - im_of<x>(w[x]) * re_of<x>(v[x]));
        });
        return acc;
    }

    // exp(+i gamma C(z)) on both states (conjugate phase table entries)
    template <int L, bool kW = false>
    static __device__ __forceinline__ void phase_dual(C2 (&v)[NE], C2 (&w)[NE], const Ctx& c, uint32_t tid, int level) {
        const TileArgs<Q>& a = *c.a;
        if constexpr (kW) {
            WA s[R], P[NP];
            const WA base = wsetup<L>(c, tid, a.wslot[level], s, P);
            const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                const C2 f = phase_tab(wat<x>(base, s, P), T);
                const real pr = re_of<x>(v[x]), pi = im_of<x>(v[x]);
                v[x] = mk<x>(pr * f.x + pi * f.y, pi * f.x - pr * f.y);
                const real lr = re_of<x>(w[x]), li = im_of<x>(w[x]);
                w[x] = mk<x>(lr * f.x + li * f.y, li * f.x - lr * f.y);
            });
            return;
        }
        int s[R];
        const int base = cut_setup<L>(c, tid, s);
        const C2* __restrict__ T = reinterpret_cast<const C2*>(a.phase) + (size_t)level * a.E1;
        for_x<NE>([&](auto X) {
            constexpr int x = decltype(X)::value;
            int cidx = base + a.crtab[L][x];
#pragma unroll
            for (int j = 0; j < R; ++j)
                if ((x >> j) & 1) cidx += s[j];
            (void)QAOA_IN_BOUNDS(a.bounds_flag, (unsigned)cidx < (unsigned)a.E1, 16u);
            const C2 f = __ldg(T + min((unsigned)cidx, (unsigned)(a.E1 - 1)));
            const real pr = re_of<x>(v[x]), pi = im_of<x>(v[x]);
            v[x] = mk<x>(pr * f.x + pi * f.y, pi * f.x - pr * f.y);
            const real lr = re_of<x>(w[x]), li = im_of<x>(w[x]);
            w[x] = mk<x>(lr * f.x + li * f.y, li * f.x - lr * f.y);
        });
    }

    // RX(2b) = [[c, -is], [-is, c]] = c * [[1, -it], [-it, 1]] with t = tan b: one FMA per
    // output component, a' = a - i t b, b' = b - i t a.  The host only hands out |t| <= 1: for
    // |tan b| > 1 it uses RX(2b) = -i X RX(2b - pi) (see coeff_kernel).  The real factors c are
    // not applied here; coeff_kernel folds them into the phase tables.  Register bits outside
    // the op's mask get t = 0, an exact identity, so the code has no data-dependent branches.
    // complex64: with N the (re, im) slot and S the (im, re) slot of a pair,
    //   N' = (t, -t) * S + N   and   S' = (-t, t) * N + S
    // as two packed FMAs (FFMA2), or, with kScalar, as the same four FMAs one lane at a time
    // (bit-identical: FFMA2 rounds each lane as one FMA).  Which is faster depends on the pass
    // (see recipe_scalar_fma).  The amplitude is the packed FMA's first factor and the
    // coefficient pair its second: in the other order the compiler keeps about one register move
    // per two FFMA2 (measured with ncu's opcode counters on a probe of 40 butterfly rounds: 0.53
    // moves per FFMA2 with the coefficient first, none with the amplitude first).
    template <bool kScalar>
    static __device__ __forceinline__ void bfly(C2& n, C2& sw, const C2 cp, const C2 cm) {
        const C2 n0 = n, s0 = sw;
        if constexpr (kScalar) {
            n = make_c2(fma(cp.x, s0.x, n0.x), fma(cp.y, s0.y, n0.y));
            sw = make_c2(fma(cm.x, n0.x, s0.x), fma(cm.y, n0.y, s0.y));
        } else {
            n = ffma2(s0, cp, n0);
            sw = ffma2(n0, cm, s0);
        }
    }
    template <int x, bool kScalar>
    static __device__ __forceinline__ void bfly_pair(C2 (&v)[NE], int j, real T, real nT) {
        const int y = x | (1 << j);
        if constexpr (kSwapOdd) {
            const C2 cp = make_c2(T, nT), cm = make_c2(nT, T);
            if constexpr (!odd_parity(x)) bfly<kScalar>(v[x], v[y], cp, cm);
            else bfly<kScalar>(v[y], v[x], cp, cm);
        } else {
            const C2 p = v[x], q = v[y];
            v[x] = make_c2(fma(T, q.y, p.x), fma(nT, q.x, p.y));
            v[y] = make_c2(fma(T, p.y, q.x), fma(nT, p.x, q.y));
        }
    }
    template <bool kFull, bool kScalar = false>
    static __device__ __forceinline__ void rx_bits(C2 (&v)[NE], uint32_t mask, real t) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const real T = (kFull || ((mask >> j) & 1u)) ? t : (real)0;
            const real nT = -T;
            for_x<NE>([&](auto X) {
                constexpr int x = decltype(X)::value;
                if (!(x & (1 << j))) bfly_pair<x, kScalar>(v, j, T, nT);
            });
        }
    }

    // RX on the register bits of a compile-time mask only (no butterflies for the other bits)
    template <uint32_t kMask, bool kScalar = false>
    static __device__ __forceinline__ void rx_fixed(C2 (&v)[NE], real t) {
        for_x<R>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if constexpr ((kMask >> j) & 1u) {
                for_x<NE>([&](auto X) {
                    constexpr int x = decltype(X)::value;
                    if constexpr (!(x & (1 << j))) bfly_pair<x, kScalar>(v, j, t, -t);
                });
            }
        });
    }

    template <bool kScalar = false>
    static __device__ __forceinline__ void rx(C2 (&v)[NE], uint32_t mask, real t) {
        if (mask == (1u << R) - 1u) rx_bits<true, kScalar>(v, mask, t);
        else rx_bits<false, kScalar>(v, mask, t);
    }

};

// Pass recipes: the op kinds of a pass program and the layouts its LOAD / SYNTH / XCHG ops
// switch to, 6 bits per op (kind | layout << 4).  A recipe instantiation of tile_kernel runs
// that program as straight-line code (levels and masks stay runtime arguments), so the register
// allocator carries the amplitudes across op boundaries and the op dispatch disappears; passes
// whose program matches no compiled recipe run the interpreting instantiation (kNops = 0).
__host__ __device__ constexpr int recipe_kind(uint64_t r, int i) { return (int)((r >> (6 * i)) & 15u); }
__host__ __device__ constexpr bool sets_layout(int kind) {
    return kind == OP_LOAD || kind == OP_SYNTH || kind == OP_XCHG;
}
// register layout in effect after op i
__host__ __device__ constexpr int recipe_layout(uint64_t r, int i) {
    int L = 0;
    for (int k = 0; k <= i; ++k)
        if (sets_layout(recipe_kind(r, k))) L = (int)((r >> (6 * k + 4)) & 3u);
    return L;
}
__host__ __device__ constexpr uint64_t recipe_step(int i, int kind, int layout) {
    return (uint64_t)(kind | (sets_layout(kind) ? layout : 0) << 4) << (6 * i);
}

struct Recipe {
    uint64_t code;    // ops 0..9
    int nops;
    uint64_t hi = 0;  // ops 10..19 (6 bits each, from bit 0)
};
// Kind and layout of op i of a program held in two words (ops 0..9 in lo, 10..19 in hi).
__host__ __device__ constexpr int recipe_kind2(uint64_t lo, uint64_t hi, int i) {
    return i < 10 ? recipe_kind(lo, i) : recipe_kind(hi, i - 10);
}
__host__ __device__ constexpr int recipe_layout2(uint64_t lo, uint64_t hi, int i) {
    int L = 0;
    for (int k = 0; k <= i; ++k)
        if (sets_layout(recipe_kind2(lo, hi, k)))
            L = (int)(((k < 10 ? lo >> (6 * k) : hi >> (6 * (k - 10))) >> 4) & 3u);
    return L;
}
// True when some op of a compiled program switches to register layout 2.
__host__ __device__ constexpr bool recipe_uses_layout2(uint64_t lo, uint64_t hi, int nops) {
    for (int i = 0; i < nops; ++i)
        if (sets_layout(recipe_kind2(lo, hi, i)) && recipe_layout2(lo, hi, i) == 2) return true;
    return false;
}

// Where a compiled program takes the CTA's cut terms K = C(o|0) and e_u (see the on-the-fly cut
// count): 1 when every op that evaluates C(z) comes after an exchange, whose barrier then
// publishes the terms warp 0 computes right after issuing its loads (no barrier of their own);
// 2 when a cut op comes first (the first pass), so that every warp computes the terms for itself
// into its own shared-memory slots (again no CTA barrier); 0 for programs without cut ops.
__host__ __device__ constexpr int recipe_cut_setup(uint64_t lo, uint64_t hi, int nops) {
    bool xchg = false, cut = false;
    for (int i = 0; i < nops; ++i) {
        const int k = recipe_kind2(lo, hi, i);
        if (k == OP_XCHG) xchg = true;
        if (k == OP_PHASE || k == OP_EXPECT || k == OP_CUTVAL || k == OP_LAMBDA || k == OP_GRADG || k == OP_PHASED) {
            if (!xchg) return 2;
            cut = true;
        }
    }
    return cut ? 1 : 0;
}

// Step i of a two-word program: in lo for i < 10, else in hi.
__host__ __device__ constexpr uint64_t recipe_step_lo(int i, int kind, int layout) {
    return i < 10 ? recipe_step(i, kind, layout) : 0;
}
__host__ __device__ constexpr uint64_t recipe_step_hi(int i, int kind, int layout) {
    return i < 10 ? 0 : recipe_step(i - 10, kind, layout);
}
// Compiled-in RX masks of a recipe, 6 bits per op (bit 5 set: the op's register mask is bits
// 0..4; clear: the mask is a runtime argument).
__host__ __device__ constexpr uint64_t fixed_mask(int i, uint32_t m) { return (uint64_t)(32u | m) << (6 * i); }
// The pass programs of the tiled plans with three or more groups (complex64 n >= 23, complex128
// n >= 20): 0 first pass, 1 group-0 pass, 2 fused boundary pass, 3 last pass, 4 complex128's
// two-exchange high-group pass.
__host__ __device__ constexpr Recipe base_recipe(int r) {
    return r == 0 ? Recipe{recipe_step(0, OP_SYNTH, 1) | recipe_step(1, OP_PHASE, 0) | recipe_step(2, OP_RX, 0) |
                               recipe_step(3, OP_XCHG, 0) | recipe_step(4, OP_RX, 0) | recipe_step(5, OP_STORE, 0),
                           6}
         : r == 1 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_XCHG, 2) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_XCHG, 0) | recipe_step(5, OP_RX, 0) |
                               recipe_step(6, OP_STORE, 0),
                           7}
         : r == 2 ? Recipe{recipe_step(0, OP_LOAD, 0) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_XCHG, 1) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_PHASE, 0) | recipe_step(5, OP_RX, 0) |
                               recipe_step(6, OP_XCHG, 0) | recipe_step(7, OP_RX, 0) | recipe_step(8, OP_STORE, 0),
                           9}
         : r == 3 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_XCHG, 0) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_EXPECT, 0) | recipe_step(5, OP_STORE, 0),
                           6}
                  : Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_XCHG, 0) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_STORE, 0),
                           5};
}
constexpr Recipe kRecipe0 = base_recipe(0), kRecipe1 = base_recipe(1), kRecipe2 = base_recipe(2),
                 kRecipe3 = base_recipe(3), kRecipe4 = base_recipe(4);
// Instantiations 5..7 are recipes 0, 2 and 3 again with every RX mask compiled in as full (the
// high-group passes of 10-bit complex64 / 8-bit complex128 groups, as at n = 33); the host
// tries them before the runtime-mask versions.
// The complex64 programs of the two-group plans (n = 15..23, and n = 24's small fused passes):
// 8 first pass, 9 fused group-0 boundary pass (13 ops: three layouts on each side of the phase),
// 10 last pass, 11 fused pass of a high group that fits one register layout, 12 last pass on
// such a group.
__host__ __device__ constexpr Recipe two_group_recipe(int r) {
    constexpr int kSteps9[13][2] = {{OP_LOAD, 0}, {OP_RX, 0}, {OP_XCHG, 2}, {OP_RX, 0}, {OP_XCHG, 1},
                                    {OP_RX, 0},   {OP_PHASE, 0}, {OP_RX, 0}, {OP_XCHG, 2}, {OP_RX, 0},
                                    {OP_XCHG, 0}, {OP_RX, 0},   {OP_STORE, 0}};
    if (r == 1) {
        Recipe d{0, 13, 0};
        for (int i = 0; i < 13; ++i) {
            d.code |= recipe_step_lo(i, kSteps9[i][0], kSteps9[i][1]);
            d.hi |= recipe_step_hi(i, kSteps9[i][0], kSteps9[i][1]);
        }
        return d;
    }
    return r == 0 ? Recipe{recipe_step(0, OP_SYNTH, 1) | recipe_step(1, OP_PHASE, 0) | recipe_step(2, OP_RX, 0) |
                               recipe_step(3, OP_XCHG, 2) | recipe_step(4, OP_RX, 0) | recipe_step(5, OP_XCHG, 0) |
                               recipe_step(6, OP_RX, 0) | recipe_step(7, OP_STORE, 0),
                           8}
         : r == 2 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_XCHG, 2) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_XCHG, 0) | recipe_step(5, OP_RX, 0) |
                               recipe_step(6, OP_EXPECT, 0) | recipe_step(7, OP_STORE, 0),
                           8}
         : r == 4 ? Recipe{recipe_step(0, OP_LOAD, 0) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_EXPECT, 0) |
                               recipe_step(3, OP_STORE, 0),
                           4}
                  : Recipe{recipe_step(0, OP_LOAD, 0) | recipe_step(1, OP_RX, 0) | recipe_step(2, OP_PHASE, 0) |
                               recipe_step(3, OP_RX, 0) | recipe_step(4, OP_STORE, 0),
                           5};
}
constexpr int kRecipes = 13;
__host__ __device__ constexpr Recipe recipe_def(int r) {
    return r >= 8 ? two_group_recipe(r - 8) : base_recipe(r == 5 ? 0 : r == 6 ? 2 : r == 7 ? 3 : r);
}
// Compiled-in masks.  The group-0 pass (recipe 1) always covers its Q bits with the same masks:
// complex64 (R = 5) layouts 1, 2, 0 take local bits 3..7, 0..2 (the layout-2 op skips bits 3, 4,
// done already), 8..12; complex128 (R = 4) takes 4..7, 0..3, 8..11.  Masks compiled in remove
// the butterflies of skipped bits and the per-bit selects, which measurably cost register moves.
template <typename real>
__host__ __device__ constexpr uint64_t recipe_masks(int r) {
    const uint32_t full = sizeof(real) == 4 ? 31u : 15u;
    if (r == 1)
        return sizeof(real) == 4 ? (fixed_mask(1, 31) | fixed_mask(3, 7) | fixed_mask(5, 31))
                                 : (fixed_mask(1, 15) | fixed_mask(3, 15) | fixed_mask(5, 15));
    if (r < 5 || r >= 8) return 0;
    const Recipe d = recipe_def(r);
    uint64_t m = 0;
    for (int i = 0; i < d.nops; ++i)
        if (recipe_kind(d.code, i) == OP_RX) m |= fixed_mask(i, full);
    return m;
}

// Complex64 recipes whose butterflies run as scalar FMAs: the first pass and the group-0 pass
// (measured at n = 33: first pass 18.4 -> 16.6 ms, group-0 pass 23.4 -> 22.9 ms).  Packed FMAs
// (FFMA2) need about 0.4-0.7 register moves each for a butterfly's old value (an FFMA2
// accumulates in place), so they save fewer instructions than they seem to; the fused boundary
// pass and the last pass are still faster packed (36.0 against 39.3 ms, 31.9 against 32.1 ms).
template <typename real>
__host__ __device__ constexpr bool recipe_scalar_fma(uint64_t recipe, int nops) {
    if (sizeof(real) != 4 || nops == 0) return false;
    for (int r : {0, 1})
        if (recipe == base_recipe(r).code && nops == base_recipe(r).nops) return true;
    return false;
}

#ifndef QAOA_TILE_MIN_BLOCKS
#define QAOA_TILE_MIN_BLOCKS 2  // resident CTAs per SM the register budget is sized for
#endif

// Resident CTAs per SM a pass kernel's register budget is sized for.  Two (128 registers a
// thread) by default; three (85) for the complex64 recipes that measured faster with 24 warps
// per SM (the first pass and the group-0 pass; at n = 33 the last pass takes 27.1 ms at two
// CTAs against 30.7 ms at three, the first pass 21.5 ms at two against 17.0 ms at three).
template <typename real, bool kW = false>
__host__ __device__ constexpr int tile_min_blocks(uint64_t recipe, int nops) {
    if (kW) return QAOA_TILE_MIN_BLOCKS;  // the weighted split needs more registers
    // (the first-pass and group-0 programs, with runtime or compiled-in masks)
    if (sizeof(real) == 4 && nops > 0)
        for (int r : {0, 1})
            if (recipe == base_recipe(r).code && nops == base_recipe(r).nops) return 3;
    return QAOA_TILE_MIN_BLOCKS;
}

// Adjoint-sweep pass programs compiled as straight-line grad_kernel instantiations: 0 the
// group-0 pass and 1 the fused boundary pass of sweeps with three or more groups (n >= 21),
// 2 the high-group pass of two-group sweeps, 3 the first pass (lambda = C psi) and 4 the last
// pass (no store) of sweeps whose high groups fit two register layouts (n = 22..28, 31..34),
// 5 the plain high-group pass of four-group sweeps (n = 31..34), 6 / 7 / 8 the first, last and
// fused boundary passes of 9-bit high groups, which need three layouts per level (n = 29, 30;
// 8 is a two-word program of 14 ops).  0..4 also run as grad_kernel instantiations, all of them
// in the persistent form (grad_pf_kernel); other programs run the interpreting instance.
__host__ __device__ constexpr Recipe grad_recipe_fused3() {
    constexpr int kSteps[14][2] = {{OP_LOAD, 0},  {OP_RXD, 0},   {OP_XCHG, 2}, {OP_RXD, 0}, {OP_XCHG, 1},
                                   {OP_RXD, 0},   {OP_GRADG, 0}, {OP_PHASED, 0}, {OP_RXD, 0}, {OP_XCHG, 2},
                                   {OP_RXD, 0},   {OP_XCHG, 0},  {OP_RXD, 0},  {OP_STORE, 0}};
    Recipe d{0, 14, 0};
    for (int i = 0; i < 14; ++i) {
        d.code |= recipe_step_lo(i, kSteps[i][0], kSteps[i][1]);
        d.hi |= recipe_step_hi(i, kSteps[i][0], kSteps[i][1]);
    }
    return d;
}
__host__ __device__ constexpr Recipe grad_recipe(int r) {
    return r == 0 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_XCHG, 2) |
                               recipe_step(3, OP_RXD, 0) | recipe_step(4, OP_XCHG, 0) | recipe_step(5, OP_RXD, 0) |
                               recipe_step(6, OP_STORE, 0),
                           7}
         : r == 1 ? Recipe{recipe_step(0, OP_LOAD, 0) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_XCHG, 1) |
                               recipe_step(3, OP_RXD, 0) | recipe_step(4, OP_GRADG, 0) | recipe_step(5, OP_PHASED, 0) |
                               recipe_step(6, OP_RXD, 0) | recipe_step(7, OP_XCHG, 0) | recipe_step(8, OP_RXD, 0) |
                               recipe_step(9, OP_STORE, 0),
                           10}
         : r == 2 ? Recipe{recipe_step(0, OP_LOAD, 0) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_GRADG, 0) |
                               recipe_step(3, OP_PHASED, 0) | recipe_step(4, OP_RXD, 0) | recipe_step(5, OP_STORE, 0),
                           6}
         : r == 3 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_LAMBDA, 0) | recipe_step(2, OP_RXD, 0) |
                               recipe_step(3, OP_XCHG, 0) | recipe_step(4, OP_RXD, 0) | recipe_step(5, OP_STORE, 0),
                           6}
         : r == 4 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_XCHG, 0) |
                               recipe_step(3, OP_RXD, 0) | recipe_step(4, OP_GRADG, 0),
                           5}
         : r == 5 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_XCHG, 0) |
                               recipe_step(3, OP_RXD, 0) | recipe_step(4, OP_STORE, 0),
                           5}
         : r == 6 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_LAMBDA, 0) | recipe_step(2, OP_RXD, 0) |
                               recipe_step(3, OP_XCHG, 2) | recipe_step(4, OP_RXD, 0) | recipe_step(5, OP_XCHG, 0) |
                               recipe_step(6, OP_RXD, 0) | recipe_step(7, OP_STORE, 0),
                           8}
         : r == 7 ? Recipe{recipe_step(0, OP_LOAD, 1) | recipe_step(1, OP_RXD, 0) | recipe_step(2, OP_XCHG, 2) |
                               recipe_step(3, OP_RXD, 0) | recipe_step(4, OP_XCHG, 0) | recipe_step(5, OP_RXD, 0) |
                               recipe_step(6, OP_GRADG, 0),
                           7}
                  : grad_recipe_fused3();
}
constexpr int kGradRecipes = 9;
// Compiled-in register masks of the sweep programs' RXD ops (6 bits per op, as recipe_masks):
// variant 1 has every RXD op full (the group-0 pass always; the fused, first and last passes of
// 8-bit high groups), variant 2 is the fused pass of 6-bit high groups, as at n = 24 (layout 1
// holds two of the group's bits), variant 3 that of 7-bit high groups (n = 25..27; three bits
// in layout 1).  Variant 0: runtime masks.
constexpr int kGradMaskVariants = 4;
__host__ __device__ constexpr uint64_t grad_masks(int r, int var) {
    uint64_t m = 0;
    if (var == 0 || r == 2 || r >= 5 || (r != 1 && var != 1)) return 0;
    const Recipe d = grad_recipe(r);
    int k = 0;
    for (int i = 0; i < d.nops; ++i)
        if (recipe_kind(d.code, i) == OP_RXD) {
            const bool mid = r == 1 && (k == 1 || k == 2);
            const uint32_t mk = (mid && var == 2) ? 0xCu : (mid && var == 3) ? 0xEu : 0xFu;
            m |= fixed_mask(i, mk);
            ++k;
        }
    return m;
}

// One pass over tile t of the state: the body of tile_kernel and tile_batch_kernel.
template <typename real, int Q, int R, bool kW, uint64_t kRecipe, int kNops, uint64_t kMasks, uint64_t kRecipeHi>
__device__ __forceinline__ void tile_body(const TileArgs<Q>& a, const uint64_t t) {
    // compiled programs that stay in layouts 0 and 1 (the high-group passes) use the swizzle with
    // immediate shared-memory offsets
    constexpr int kSw = (kNops > 0 && !recipe_uses_layout2(kRecipe, kRecipeHi, kNops)) ? 1 : 0;
    using T = Tile<real, Q, R, true, kSw>;
    using C2 = typename T::C2;
    using WA = typename T::WA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // CTA cut terms: one copy, or one per warp when every warp computes its own (kSetup == 2)
    constexpr int kSetup = (!kW && kNops > 0) ? recipe_cut_setup(kRecipe, kRecipeHi, kNops) : -1;
    constexpr int kCopies = kSetup == 2 ? T::NT / 32 : 1;
    __shared__ int sE_all[kCopies][Q];
    __shared__ int sK_all[kCopies];

    __shared__ WA sKw[kW ? kWSlots : 1];
    __shared__ WA sEw[kW ? kWSlots : 1][Q];

    unsigned char* tile = smem_raw;
    const uint32_t tid = threadIdx.x;
    uint64_t zb = 0;  // outer index bits of tile t: runs of tile-id bits deposited in place
    for (int r = 0; r < a.nruns; ++r) zb |= ((t >> a.run_src[r]) & ((1ull << a.run_len[r]) - 1ull)) << a.run_dst[r];

    const uint32_t wcopy = kSetup == 2 ? tid / 32 : 0;
    int* const sE = sE_all[wcopy];
    // K = C(o|0) by Algorithm 3 (one popcount per vertex, over a warp) and the e_u terms of the
    // tile's local bits, by the calling warp into copy `wcopy`
    auto cut_terms = [&]() {
        const uint32_t lane = tid & 31u;
        int acc = 0;
        for (int v = (int)lane; v < a.n; v += 32) {
            const uint64_t bI = 0ull - ((zb >> v) & 1ull);
            acc += __popcll(a.gmask[v] & (bI ^ zb));
        }
        acc = warp_sum_int(acc);
        if (lane == 0) sK_all[wcopy] = acc;
        if (lane < (uint32_t)Q) sE[lane] = __popcll(a.outAdj[lane]) - 2 * __popcll(a.outAdj[lane] & zb);
    };
    if constexpr (kW) {
        if (a.need_cut) weighted_cta_setup<WA, Q>(a, zb, sKw, sEw, tid, T::NT);
    } else if constexpr (kSetup == 2) {
        if (a.need_cut) cut_terms();
        __syncwarp();
    } else if constexpr (kSetup < 0) {  // interpreting program: the terms before any op
        if (a.need_cut) {
            if (tid < 32) cut_terms();
            __syncthreads();
        }
    }

    typename T::Ctx c;
    c.zb = zb;
    c.K = (!kW && (kSetup == 2 || kSetup < 0) && a.need_cut) ? sK_all[wcopy] : 0;
    c.a = &a;
    c.sE = sE;
    c.wK = sKw;
    c.wE = sEw;
    const bool podd = ((__popcll(zb) + __popc(tid)) & 1) != 0;  // P of the parity form
    c.sg = (T::kSwapOdd && podd) ? (real)-1 : (real)1;

    C2 v[T::NE];
    int L = 0;
    double accC = 0.0, accN = 0.0;
    bool did_expect = false;

    if constexpr (kNops > 0) {
        const C2* mix = reinterpret_cast<const C2*>(a.mix);
        T::template for_x<kNops>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int kind = recipe_kind2(kRecipe, kRecipeHi, i);
            constexpr int Lc = recipe_layout2(kRecipe, kRecipeHi, i);
            constexpr int Lp = i == 0 ? 0 : recipe_layout2(kRecipe, kRecipeHi, i - 1);
            if constexpr (kind == OP_SYNTH) {
                const real amp = (real)a.init_amp;
                T::template for_x<T::NE>([&](auto X) {
                    constexpr int x = decltype(X)::value;
                    const bool sw = T::kSwapOdd && (odd_parity(x) != podd);
                    v[x] = make_c2(sw ? (real)0 : amp, sw ? amp : (real)0);
                });
            } else if constexpr (kind == OP_LOAD) {
                T::template load<Lc>(v, c, tid);
            } else if constexpr (kind == OP_XCHG) {
                // no barrier before the writes: a thread writes exactly the tile positions it read
                // in the previous exchange, or the tile is still unused (see to_smem)
                T::template to_smem<Lp>(v, tile, tid, a.bounds_flag);
                __syncthreads();
                T::template from_smem<Lc>(v, tile, tid, a.bounds_flag);
            } else if constexpr (kind == OP_RX) {
                const Op op = a.ops[i];
                constexpr uint32_t fm = i < 10 ? (uint32_t)((kMasks >> (6 * i)) & 63u) : 0u;
                constexpr bool kScalar = recipe_scalar_fma<real>(kRecipe, kNops);
                if constexpr ((fm & 32u) != 0)
                    T::template rx_fixed<(fm & 31u), kScalar>(v, c.sg * mix[3 * op.arg + 1].x);
                else
                    T::template rx<kScalar>(v, op.mask, c.sg * mix[3 * op.arg + 1].x);
            } else if constexpr (kind == OP_PHASE) {
                if constexpr (kSetup == 1) c.K = sK_all[0];
                T::template phase<Lc, kW>(v, c, tid, a.ops[i].arg);
            } else if constexpr (kind == OP_EXPECT) {
                did_expect = true;
                if constexpr (kSetup == 1) c.K = sK_all[0];
                T::template expect<Lc, kW>(v, c, tid, accC, accN);
            } else if constexpr (kind == OP_CUTVAL) {
                if constexpr (kSetup == 1) c.K = sK_all[0];
                T::template cutval<Lc, kW>(c, tid);
            } else if constexpr (kind == OP_STORE) {
                T::template store<Lc>(v, c, tid);
            }
            // after the first op (its loads in flight), warp 0 computes the cut terms; the next
            // exchange's barrier publishes them.  Programs without cut ops run with need_cut = 0
            // and keep the (never taken) branch: it ends the load block, so that every warp
            // issues all of its loads before its first butterfly (the group-0 pass at n = 33:
            // 22.7 ms without it, 21.1 ms with it)
            if constexpr ((kSetup == 1 || kSetup == 0) && i == 0)
                if (a.need_cut && tid < 32) cut_terms();
        });
    }
    for (int i = 0; kNops == 0 && i < a.nops; ++i) {
        const Op op = a.ops[i];
        switch (op.kind) {
            case OP_SYNTH: {  // |+>^n in the parity form: (amp, 0), or (0, amp) where swapped
                const real amp = (real)a.init_amp;
                T::template for_x<T::NE>([&](auto X) {
                    constexpr int x = decltype(X)::value;
                    const bool sw = T::kSwapOdd && (odd_parity(x) != podd);
                    v[x] = make_c2(sw ? (real)0 : amp, sw ? amp : (real)0);
                });
                L = op.layout;
                break;
            }
            case OP_LOAD:
                L = op.layout;
                if (L == 0) T::template load<0>(v, c, tid);
                else if (L == 1) T::template load<1>(v, c, tid);
                else T::template load<2>(v, c, tid);
                break;
            case OP_XCHG:
                if (L == 0) T::template to_smem<0>(v, tile, tid, a.bounds_flag);
                else if (L == 1) T::template to_smem<1>(v, tile, tid, a.bounds_flag);
                else T::template to_smem<2>(v, tile, tid, a.bounds_flag);
                __syncthreads();
                L = op.layout;
                if (L == 0) T::template from_smem<0>(v, tile, tid, a.bounds_flag);
                else if (L == 1) T::template from_smem<1>(v, tile, tid, a.bounds_flag);
                else T::template from_smem<2>(v, tile, tid, a.bounds_flag);
                break;
            case OP_RX:
                T::rx(v, op.mask, c.sg * reinterpret_cast<const C2*>(a.mix)[3 * op.arg + 1].x);
                break;
            case OP_PHASE:
                if (L == 0) T::template phase<0, kW>(v, c, tid, op.arg);
                else if (L == 1) T::template phase<1, kW>(v, c, tid, op.arg);
                else T::template phase<2, kW>(v, c, tid, op.arg);
                break;
            case OP_EXPECT:
                did_expect = true;
                if (L == 0) T::template expect<0, kW>(v, c, tid, accC, accN);
                else if (L == 1) T::template expect<1, kW>(v, c, tid, accC, accN);
                else T::template expect<2, kW>(v, c, tid, accC, accN);
                break;
            case OP_CUTVAL:
                if (L == 0) T::template cutval<0, kW>(c, tid);
                else if (L == 1) T::template cutval<1, kW>(c, tid);
                else T::template cutval<2, kW>(c, tid);
                break;
            case OP_STORE:
                if (L == 0) T::template store<0>(v, c, tid);
                else if (L == 1) T::template store<1>(v, c, tid);
                else T::template store<2>(v, c, tid);
                break;
            default:
                break;
        }
    }

    if (did_expect) {
        // FP64 sums by warp 0 alone (FP64 adds issue at 1/64 of the FP32 rate here), through
        // the tile buffer once every thread is past its last exchange
        double* red = reinterpret_cast<double*>(tile);
        __syncthreads();
        red[tid] = accC;
        red[T::NT + tid] = accN;
        __syncthreads();
        if (tid < 32) {
            double sc = 0.0, sn = 0.0;
#pragma unroll
            for (int i = 0; i < T::NT / 32; ++i) {
                sc += red[tid + 32 * i];
                sn += red[T::NT + tid + 32 * i];
            }
            sc = warp_sum_double(sc);
            sn = warp_sum_double(sn);
            if (tid == 0) a.partials[t] = make_double2(sc, sn);
        }
    }
}

template <typename real, int Q, int R, bool kW, uint64_t kRecipe = 0, int kNops = 0, uint64_t kMasks = 0,
          uint64_t kRecipeHi = 0>
__global__ void __launch_bounds__(1 << (Q - R), tile_min_blocks<real, kW>(kRecipe, kNops))
    tile_kernel(const __grid_constant__ TileArgs<Q> a) {
    tile_body<real, Q, R, kW, kRecipe, kNops, kMasks, kRecipeHi>(a, blockIdx.x);
}

// The same pass for blockIdx.y of several requests of one shape (the request server's packed
// launches of mid-size states): request y's arguments are copied from args[y] into shared memory
// first, so one launch covers every tile of every request.
template <typename real, int Q, int R, bool kW, uint64_t kRecipe = 0, int kNops = 0, uint64_t kMasks = 0,
          uint64_t kRecipeHi = 0>
__global__ void __launch_bounds__(1 << (Q - R), tile_min_blocks<real, kW>(kRecipe, kNops))
    tile_batch_kernel(const TileArgs<Q>* __restrict__ args) {
    __shared__ __align__(16) TileArgs<Q> sa;
    static_assert(sizeof(TileArgs<Q>) % 16 == 0, "TileArgs is copied in 16-byte words");
    const uint4* src = reinterpret_cast<const uint4*>(args + blockIdx.y);
    uint4* dst = reinterpret_cast<uint4*>(&sa);
    for (uint32_t i = threadIdx.x; i < sizeof(TileArgs<Q>) / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    tile_body<real, Q, R, kW, kRecipe, kNops, kMasks, kRecipeHi>(sa, blockIdx.x);
}

// ---------------------------------------------------------------------------------- adjoint sweep

// One pass of the adjoint sweep over psi (a.state) and lambda (a.state2), same tiling as
// tile_kernel.  Per CTA it writes, for accumulator slots 0 and 1, (sum of RXD pair terms,
// sum of GRADG terms) to partials[2 t + slot].
// (complex64 holds both states in 64 registers and runs two CTAs per SM; complex128 needs 128)
template <typename real, int Q, int R, bool kW, uint64_t kRecipe = 0, int kNops = 0, uint64_t kMasks = 0>
__global__ void __launch_bounds__(1 << (Q - R), sizeof(real) == 4 ? 2 : 1) grad_kernel(const __grid_constant__ TileArgs<Q> a) {
    // complex64: both states in the forward passes' parity form, packed butterflies with the real
    // factors undone through a.gpow and the sweep's phase tables; complex128: plain form, exact
    // RX(2 beta)^dagger butterflies
    constexpr bool kPG = sizeof(real) == 4;
    constexpr bool kSweepScalar = false;
    using T = Tile<real, Q, R, kPG>;
    using C2 = typename T::C2;
    using WA = typename T::WA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the CTA's cut terms, placed as in tile_body (kSetup: see recipe_cut_setup)
    constexpr int kSetup = (!kW && kNops > 0) ? recipe_cut_setup(kRecipe, 0, kNops) : -1;
    constexpr int kCopies = kSetup == 2 ? T::NT / 32 : 1;
    __shared__ int sE_all[kCopies][Q];
    __shared__ int sK_all[kCopies];

    __shared__ WA sKw[kW ? kWSlots : 1];
    __shared__ WA sEw[kW ? kWSlots : 1][Q];

    // psi and lambda exchange through one tile each
    unsigned char* tile = smem_raw;
    unsigned char* tile2 = smem_raw + (1u << Q) * sizeof(C2);
    const uint32_t tid = threadIdx.x;
    const uint64_t t = blockIdx.x;
    uint64_t zb = 0;
    for (int r = 0; r < a.nruns; ++r) zb |= ((t >> a.run_src[r]) & ((1ull << a.run_len[r]) - 1ull)) << a.run_dst[r];
    const uint32_t wcopy = kSetup == 2 ? tid / 32 : 0;
    int* const sE = sE_all[wcopy];
    auto cut_terms = [&]() {
        const uint32_t lane = tid & 31u;
        int acc = 0;
        for (int v = (int)lane; v < a.n; v += 32) {
            const uint64_t bI = 0ull - ((zb >> v) & 1ull);
            acc += __popcll(a.gmask[v] & (bI ^ zb));
        }
        acc = warp_sum_int(acc);
        if (lane == 0) sK_all[wcopy] = acc;
        if (lane < (uint32_t)Q) sE[lane] = __popcll(a.outAdj[lane]) - 2 * __popcll(a.outAdj[lane] & zb);
    };
    if constexpr (kW) {
        weighted_cta_setup<WA, Q>(a, zb, sKw, sEw, tid, T::NT);
        __syncthreads();
    } else if constexpr (kSetup == 2) {
        cut_terms();
        __syncwarp();
    } else if constexpr (kSetup < 0) {
        if (tid < 32) cut_terms();
        __syncthreads();
    }
    typename T::Ctx c;
    c.zb = zb;
    c.K = (!kW && (kSetup == 2 || kSetup < 0)) ? sK_all[wcopy] : 0;
    c.a = &a;
    c.sE = sE;
    c.wK = sKw;
    c.wE = sEw;
    c.sg = (kPG && (((__popcll(zb) + __popc(tid)) & 1) != 0)) ? (real)-1 : (real)1;  // P of the parity form

    C2 v[T::NE], w[T::NE];
    int L = 0;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // (pair terms, gamma terms) for slots 0 and 1
    const bool lam_init = a.nops > 1 && a.ops[1].kind == OP_LAMBDA;
    // d/d beta pair terms of one RXD op (and its butterflies), as a true-scale FP64 sum
    auto rxd_op = [&](auto FM, const Op& op, C2(&vv)[T::NE], C2(&ww)[T::NE]) -> double {
        const int level = sweep_level(op.arg);
        if constexpr (kPG) {
            const real t = reinterpret_cast<const C2*>(a.mix)[3 * level + 1].x;
            const real d = T::template rxd_parity<kSweepScalar, decltype(FM)::value>(vv, ww, op.mask, -c.sg * t);
            return (double)(c.sg * d) * a.gpow[level * (kMaxN + 1) + sweep_done(op.arg)];
        } else {
            const C2 cs = reinterpret_cast<const C2*>(a.mix)[3 * level];
            return (double)T::rx_dual(vv, ww, op.mask, cs.x, cs.y);
        }
    };
    // d/d gamma terms of one GRADG op (after all n butterflies of its level), true scale
    auto gradg_op = [&](auto Lt, const Op& op, const C2(&vv)[T::NE], const C2(&ww)[T::NE]) -> double {
        constexpr int Lx = decltype(Lt)::value;
        if constexpr (kPG) {
            const real g = T::template grad_gamma_parity<Lx, kW>(vv, ww, c, tid);
            return (double)(c.sg * g) * a.gpow[sweep_level(op.arg) * (kMaxN + 1) + a.n];
        } else {
            return (double)T::template grad_gamma<Lx, kW>(vv, ww, c, tid);
        }
    };

#define QAOA_BY_LAYOUT(F, ...)                     \
    do {                                           \
        if (L == 0) T::template F<0>(__VA_ARGS__); \
        else if (L == 1) T::template F<1>(__VA_ARGS__); \
        else T::template F<2>(__VA_ARGS__);        \
    } while (0)

    if constexpr (kNops > 0) {  // a compiled program: kinds and layouts are template constants
        T::template for_x<kNops>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int kind = recipe_kind(kRecipe, i);
            constexpr int Lc = recipe_layout(kRecipe, i);
            constexpr int Lp = i == 0 ? 0 : recipe_layout(kRecipe, i - 1);
            if constexpr (kind == OP_LOAD) {
                T::template load_from<Lc>(v, c, tid, a.state);
                // the sweep's first pass makes lambda from psi instead of loading it
                if constexpr (!(kNops > 1 && recipe_kind(kRecipe, 1) == OP_LAMBDA))
                    T::template load_from<Lc>(w, c, tid, a.state2);
            } else if constexpr (kind == OP_LAMBDA) {
                T::template lambda_init<Lc, kW>(v, w, c, tid);
            } else if constexpr (kind == OP_XCHG) {
                // one barrier: a thread writes exactly the positions it read in the previous
                // exchange (see to_smem)
                T::template to_smem<Lp>(v, tile, tid, a.bounds_flag);
                T::template to_smem<Lp>(w, tile2, tid, a.bounds_flag);
                __syncthreads();
                T::template from_smem<Lc>(v, tile, tid, a.bounds_flag);
                T::template from_smem<Lc>(w, tile2, tid, a.bounds_flag);
            } else if constexpr (kind == OP_RXD) {
                const Op op = a.ops[i];
                constexpr uint32_t fm = i < 10 ? (uint32_t)((kMasks >> (6 * i)) & 63u) : 0u;
                const double d = rxd_op(std::integral_constant<uint32_t, fm>{}, op, v, w);
                if (sweep_slot(op.arg)) acc[2] += d;
                else acc[0] += d;
            } else if constexpr (kind == OP_GRADG) {
                if constexpr (kSetup == 1) c.K = sK_all[0];
                const double d = gradg_op(std::integral_constant<int, Lc>{}, a.ops[i], v, w);
                if (sweep_slot(a.ops[i].arg)) acc[3] += d;
                else acc[1] += d;
            } else if constexpr (kind == OP_PHASED) {
                if constexpr (kSetup == 1) c.K = sK_all[0];
                if constexpr (kPG) T::template phase_dual_parity<Lc, kW>(v, w, c, tid, a.ops[i].arg);
                else T::template phase_dual<Lc, kW>(v, w, c, tid, a.ops[i].arg);
            } else if constexpr (kind == OP_STORE) {
                T::template store_to<Lc>(v, c, tid, a.state);
                T::template store_to<Lc>(w, c, tid, a.state2);
            }
            // after the loads, warp 0 computes the cut terms; the next exchange's barrier
            // publishes them (as in tile_body, the branch also ends the load block)
            if constexpr ((kSetup == 1 || kSetup == 0) && i == 0)
                if (a.need_cut && tid < 32) cut_terms();
        });
    }
    for (int i = 0; kNops == 0 && i < a.nops; ++i) {
        const Op op = a.ops[i];
        switch (op.kind) {
            case OP_LOAD:
                L = op.layout;
                QAOA_BY_LAYOUT(load_from, v, c, tid, a.state);
                if (!lam_init) QAOA_BY_LAYOUT(load_from, w, c, tid, a.state2);
                break;
            case OP_LAMBDA:
                if (L == 0) T::template lambda_init<0, kW>(v, w, c, tid);
                else if (L == 1) T::template lambda_init<1, kW>(v, w, c, tid);
                else T::template lambda_init<2, kW>(v, w, c, tid);
                break;
            case OP_XCHG:
                QAOA_BY_LAYOUT(to_smem, v, tile, tid, a.bounds_flag);
                QAOA_BY_LAYOUT(to_smem, w, tile2, tid, a.bounds_flag);
                __syncthreads();
                L = op.layout;
                QAOA_BY_LAYOUT(from_smem, v, tile, tid, a.bounds_flag);
                QAOA_BY_LAYOUT(from_smem, w, tile2, tid, a.bounds_flag);
                break;
            case OP_RXD:
                acc[2 * sweep_slot(op.arg)] += rxd_op(std::integral_constant<uint32_t, 0>{}, op, v, w);
                break;
            case OP_GRADG: {
                double g = 0;
                if (L == 0) g = gradg_op(std::integral_constant<int, 0>{}, op, v, w);
                else if (L == 1) g = gradg_op(std::integral_constant<int, 1>{}, op, v, w);
                else g = gradg_op(std::integral_constant<int, 2>{}, op, v, w);
                acc[2 * sweep_slot(op.arg) + 1] += g;
                break;
            }
            case OP_PHASED:
                if constexpr (kPG) {
                    if (L == 0) T::template phase_dual_parity<0, kW>(v, w, c, tid, op.arg);
                    else if (L == 1) T::template phase_dual_parity<1, kW>(v, w, c, tid, op.arg);
                    else T::template phase_dual_parity<2, kW>(v, w, c, tid, op.arg);
                } else {
                    if (L == 0) T::template phase_dual<0, kW>(v, w, c, tid, op.arg);
                    else if (L == 1) T::template phase_dual<1, kW>(v, w, c, tid, op.arg);
                    else T::template phase_dual<2, kW>(v, w, c, tid, op.arg);
                }
                break;
            case OP_STORE:
                L = op.layout;
                QAOA_BY_LAYOUT(store_to, v, c, tid, a.state);
                QAOA_BY_LAYOUT(store_to, w, c, tid, a.state2);
                break;
            default:
                break;
        }
    }
#undef QAOA_BY_LAYOUT
    // summed in FP64 by warp 0 alone, through the tile buffer once every thread is past its
    // last exchange
    double* red = reinterpret_cast<double*>(tile);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k * T::NT + tid] = acc[k];
    __syncthreads();
    if (tid < 32) {
        double r[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < T::NT / 32; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] += red[k * T::NT + tid + 32 * i];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = warp_sum_double(r[k]);
        if (tid == 0) {
            a.partials[2 * t] = make_double2(r[0], r[1]);
            a.partials[2 * t + 1] = make_double2(r[2], r[3]);
        }
    }
}

// Whether a compiled (one- or two-word) program has an op of the given kind.
__host__ __device__ constexpr bool recipe_has(uint64_t lo, uint64_t hi, int nops, int kind) {
    for (int i = 0; i < nops; ++i)
        if (recipe_kind2(lo, hi, i) == kind) return true;
    return false;
}

// Index of the last exchange of a compiled (one- or two-word) program (-1: none).
__host__ __device__ constexpr int recipe_last_xchg(uint64_t lo, uint64_t hi, int nops) {
    int last = -1;
    for (int i = 0; i < nops; ++i)
        if (recipe_kind2(lo, hi, i) == OP_XCHG) last = i;
    return last;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The compiled complex64 sweep programs (unit or edge weights) as a persistent, prefetching kernel: CTA b
// runs tiles b, b + G, b + 2G, ... (G = gridDim.x, at most the CTAs that fit the GPU at once).
// The next tile's lambda (psi in the first pass, which makes lambda itself) is copied into its
// exchange tile by cp.async as soon as the program's last exchange has read it, so the copy
// overlaps the rest of the current tile (its last butterflies and its stores); the program's
// LOAD then reads lambda from shared memory and psi straight from HBM.  (Staging both states
// moved the passes' top stall to the shared-memory queue: 2.5-3 % slower, except in the fused
// boundary passes, which stage both.)  The FP64 sums of a thread run over all of its tiles and each CTA writes one partial
// pair per slot: partials[2 b + slot] for b < G (the host reduces G entries per pass).  The
// order is fixed for a given grid, so results are deterministic; they equal grad_kernel's up to
// the order of the per-tile sums.
template <int Q, int R, bool kW, uint64_t kRecipe, int kNops, uint64_t kMasks, uint64_t kRecipeHi = 0>
__global__ void __launch_bounds__(1 << (Q - R), 2)
    grad_pf_kernel(const __grid_constant__ TileArgs<Q> a, uint64_t tiles) {
    using real = float;
    using T = Tile<real, Q, R, true>;
    using C2 = typename T::C2;
    using WA = typename T::WA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // unit weights: where the CTA's cut terms are computed (recipe_cut_setup); edge weights: the
    // weighted terms of every tile by all threads (weighted_cta_setup), -1
    constexpr int kSetup = kW ? -1 : recipe_cut_setup(kRecipe, kRecipeHi, kNops);
    static_assert(kSetup >= -1 && kSetup <= 2, "compiled sweep program");
    // cut terms: one copy per warp (kSetup 2), else two copies used by alternate tiles, so that
    // a tile's terms can be written while slower warps still read the previous tile's
    constexpr int kCopies = kSetup == 2 ? T::NT / 32 : 2;
    __shared__ int sE_all[kW ? 1 : kCopies][Q];
    __shared__ int sK_all[kW ? 1 : kCopies];
    __shared__ WA sKw[kW ? 2 : 1][kWSlots];
    __shared__ WA sEw[kW ? 2 : 1][kWSlots][Q];
    constexpr bool kLam = kNops > 1 && recipe_kind2(kRecipe, kRecipeHi, 1) == OP_LAMBDA;
    constexpr int kLastX = recipe_last_xchg(kRecipe, kRecipeHi, kNops);
    static_assert(kLastX > 0, "the prefetch follows the program's last exchange");
    constexpr int kL0 = recipe_layout2(kRecipe, kRecipeHi, 0);
    // the fused boundary programs (with the inverse phase) stage psi as well: measured faster
    // for them (2.24 against 2.29 ms per pass at n = 28), slower for the others
    constexpr bool kBoth = !kLam && recipe_has(kRecipe, kRecipeHi, kNops, OP_PHASED);

    unsigned char* tile = smem_raw;
    unsigned char* tile2 = smem_raw + (1u << Q) * sizeof(C2);
    const uint32_t tid = threadIdx.x;
    auto zb_of = [&](uint64_t t) {
        uint64_t z = 0;
        for (int r = 0; r < a.nruns; ++r) z |= ((t >> a.run_src[r]) & ((1ull << a.run_len[r]) - 1ull)) << a.run_dst[r];
        return z;
    };
    typename T::Ctx c;
    c.a = &a;
    c.wK = nullptr;
    c.wE = nullptr;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // (pair terms, gamma terms) for slots 0 and 1

    auto prefetch = [&](uint64_t t) {
        typename T::Ctx cn = c;
        cn.zb = zb_of(t);
        // lambda is staged (psi in the first pass, which makes lambda; both in fused passes)
        if constexpr (kLam || kBoth) T::template prefetch_to<kL0>(tile, cn, tid, a.state, a.bounds_flag);
        if constexpr (!kLam) T::template prefetch_to<kL0>(tile2, cn, tid, a.state2, a.bounds_flag);
        cp_async_commit();
    };
    if ((uint64_t)blockIdx.x < tiles) prefetch(blockIdx.x);

    int it = 0;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
        const uint64_t zb = zb_of(t);
        const uint32_t copy = kW ? 0u : (kSetup == 2 ? tid / 32 : (uint32_t)(it & 1));
        int* const sE = sE_all[copy];
        auto cut_terms = [&]() {
            const uint32_t lane = tid & 31u;
            int s = 0;
            for (int v = (int)lane; v < a.n; v += 32) {
                const uint64_t bI = 0ull - ((zb >> v) & 1ull);
                s += __popcll(a.gmask[v] & (bI ^ zb));
            }
            s = warp_sum_int(s);
            if (lane == 0) sK_all[copy] = s;
            if (lane < (uint32_t)Q) sE[lane] = __popcll(a.outAdj[lane]) - 2 * __popcll(a.outAdj[lane] & zb);
        };
        c.zb = zb;
        c.sE = sE;
        c.sg = (((__popcll(zb) + __popc(tid)) & 1) != 0) ? (real)-1 : (real)1;  // P of the parity form
        cp_async_wait_all();
        __syncthreads();  // every thread's copies of tile t have landed
        if constexpr (kW) {
            weighted_cta_setup<WA, Q>(a, zb, sKw[it & 1], sEw[it & 1], tid, T::NT);
            c.wK = sKw[it & 1];
            c.wE = sEw[it & 1];
            c.K = 0;
        } else if constexpr (kSetup == 2) {
            cut_terms();
            __syncwarp();
            c.K = sK_all[copy];
        } else {
            c.K = 0;
        }
        C2 v[T::NE], w[T::NE];
        T::template for_x<kNops>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int kind = recipe_kind2(kRecipe, kRecipeHi, i);
            constexpr int Lc = recipe_layout2(kRecipe, kRecipeHi, i);
            constexpr int Lp = i == 0 ? 0 : recipe_layout2(kRecipe, kRecipeHi, i - 1);
            if constexpr (kind == OP_LOAD) {
                if constexpr (kLam || kBoth) T::template from_smem<Lc>(v, tile, tid, a.bounds_flag);
                else T::template load_from<Lc>(v, c, tid, a.state);  // psi straight from HBM
                if constexpr (!kLam) T::template from_smem<Lc>(w, tile2, tid, a.bounds_flag);
            } else if constexpr (kind == OP_LAMBDA) {
                T::template lambda_init<Lc, kW>(v, w, c, tid);
            } else if constexpr (kind == OP_XCHG) {
                T::template to_smem<Lp>(v, tile, tid, a.bounds_flag);
                T::template to_smem<Lp>(w, tile2, tid, a.bounds_flag);
                __syncthreads();
                T::template from_smem<Lc>(v, tile, tid, a.bounds_flag);
                T::template from_smem<Lc>(w, tile2, tid, a.bounds_flag);
                if constexpr (i == kLastX) {
                    __syncthreads();  // the tiles are read: the next tile may land in them
                    if (t + gridDim.x < tiles) prefetch(t + gridDim.x);
                }
            } else if constexpr (kind == OP_RXD) {
                const Op op = a.ops[i];
                constexpr uint32_t fm = i < 10 ? (uint32_t)((kMasks >> (6 * i)) & 63u) : 0u;
                const int level = sweep_level(op.arg);
                const real tt = reinterpret_cast<const C2*>(a.mix)[3 * level + 1].x;
                const real d = T::template rxd_parity<false, fm>(v, w, op.mask, -c.sg * tt);
                const double dd = (double)(c.sg * d) * a.gpow[level * (kMaxN + 1) + sweep_done(op.arg)];
                if (sweep_slot(op.arg)) acc[2] += dd;
                else acc[0] += dd;
            } else if constexpr (kind == OP_GRADG) {
                if constexpr (kSetup == 1) c.K = sK_all[copy];
                // a GRADG directly followed by the PHASED of the same layout runs as one op
                constexpr bool kMerged = !kW && i + 1 < kNops && recipe_kind2(kRecipe, kRecipeHi, i + 1) == OP_PHASED;
                real g;
                if constexpr (kMerged) g = T::template grad_gamma_phase_dual_parity<Lc>(v, w, c, tid, a.ops[i + 1].arg);
                else g = T::template grad_gamma_parity<Lc, kW>(v, w, c, tid);
                const double dd = (double)(c.sg * g) * a.gpow[sweep_level(a.ops[i].arg) * (kMaxN + 1) + a.n];
                if (sweep_slot(a.ops[i].arg)) acc[3] += dd;
                else acc[1] += dd;
            } else if constexpr (kind == OP_PHASED) {
                constexpr bool kMerged = !kW && i > 0 && recipe_kind2(kRecipe, kRecipeHi, i - 1) == OP_GRADG;
                if constexpr (!kMerged) {
                    if constexpr (kSetup == 1) c.K = sK_all[copy];
                    T::template phase_dual_parity<Lc, kW>(v, w, c, tid, a.ops[i].arg);
                }
            } else if constexpr (kind == OP_STORE) {
                T::template store_to<Lc>(v, c, tid, a.state);
                T::template store_to<Lc>(w, c, tid, a.state2);
            }
            // warp 0 computes the cut terms after its loads; the next exchange's barrier
            // publishes them
            if constexpr (!kW && kSetup == 1 && i == 0)
                if (a.need_cut && tid < 32) cut_terms();
        });
    }
    // one partial pair per slot and CTA, summed in FP64 by warp 0 through the (now idle) tile
    double* red = reinterpret_cast<double*>(tile);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k * T::NT + tid] = acc[k];
    __syncthreads();
    if (tid < 32) {
        double r[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < T::NT / 32; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] += red[k * T::NT + tid + 32 * i];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = warp_sum_double(r[k]);
        if (tid == 0 && (uint64_t)blockIdx.x < tiles) {
            a.partials[2 * blockIdx.x] = make_double2(r[0], r[1]);
            a.partials[2 * blockIdx.x + 1] = make_double2(r[2], r[3]);
        }
    }
}

// A batch of adjoint passes whose partials are reduced by one launch: pass i of the batch wrote
// cnt[i] partial pairs at partials + 2 tiles i, and its slots belong to levels lev[i][0..1].
constexpr int kGradBatchMax = 64;
struct GradBatch {
    int npass;
    int lev[kGradBatchMax][2];
    uint32_t cnt[kGradBatchMax];  // partial pairs pass i wrote (its tiles, or its CTAs)
};

// The per-level sums of a batch of passes: CTA i sums pass i's partials exactly as
// grad_reduce_kernel does and leaves the four sums in acc[2p + 4i ..]; the CTA that finishes last
// (a ticket counter at acc[2p + 4 kGradBatchMax], zero on entry and left zero) adds them to the
// per-level sums in pass order, so the result is bit-identical to one grad_reduce_kernel launch
// after each pass.  No CTA waits for another.
static __global__ void __launch_bounds__(1024) grad_reduce_batch_kernel(const double2* __restrict__ partials,
                                                                 uint64_t tiles, const __grid_constant__ GradBatch b,
                                                                 int p, double* __restrict__ acc) {
    __shared__ double sm[4][1024];
    __shared__ bool last;
    const double2* pp = partials + (size_t)blockIdx.x * 2 * tiles;
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint64_t i = threadIdx.x; i < b.cnt[blockIdx.x]; i += 1024) {
        const double2 a = pp[2 * i], c = pp[2 * i + 1];
        r[0] += a.x;
        r[1] += a.y;
        r[2] += c.x;
        r[3] += c.y;
    }
    for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    double* sums = acc + 2 * p;
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(acc + 2 * p + 4 * kGradBatchMax);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) sums[4 * blockIdx.x + k] = sm[k][0];
        __threadfence();
        last = atomicAdd(ticket, 1ull) == (unsigned long long)gridDim.x - 1ull;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        for (int i = 0; i < b.npass; ++i) {
            const double s0 = __ldcg(sums + 4 * i), s1 = __ldcg(sums + 4 * i + 1);
            const double s2 = __ldcg(sums + 4 * i + 2), s3 = __ldcg(sums + 4 * i + 3);
            if (b.lev[i][0] >= 0) {
                acc[b.lev[i][0]] += s0;
                acc[p + b.lev[i][0]] += s1;
            }
            if (b.lev[i][1] >= 0) {
                acc[b.lev[i][1]] += s2;
                acc[p + b.lev[i][1]] += s3;
            }
        }
        *ticket = 0ull;
    }
}

// Adds, in a fixed order, the per-tile adjoint partials of one pass to the per-level sums:
// slot s of the pass belongs to level lev[s] (-1: unused); acc[level] gets the pair terms
// (d/d beta) and acc[p + level] the gamma terms.
static __global__ void __launch_bounds__(1024) grad_reduce_kernel(const double2* __restrict__ partials, uint64_t tiles,
                                                           int lev0, int lev1, int p, double* __restrict__ acc) {
    __shared__ double sm[4][1024];
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint64_t i = threadIdx.x; i < tiles; i += 1024) {
        const double2 a = partials[2 * i], b = partials[2 * i + 1];
        r[0] += a.x;
        r[1] += a.y;
        r[2] += b.x;
        r[3] += b.y;
    }
    for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (lev0 >= 0) {
            acc[lev0] += sm[0][0];
            acc[p + lev0] += sm[1][0];
        }
        if (lev1 >= 0) {
            acc[lev1] += sm[2][0];
            acc[p + lev1] += sm[3][0];
        }
    }
}

// Whole-state adjoint sweep for small n (psi and lambda both in shared memory, one CTA).
struct SmallGradJob {
    int32_t n, levels, E1;
    uint64_t gmask[kMaxN];
    const void* state;   // psi after the forward levels
    const void* phase;   // plain tables [level][E1]
    const void* mix;     // [3 * level]: (cos b, sin b)
    double* acc;         // [2 * levels]: pair sums, gamma sums
    const void* wfix;    // edge-weighted graphs: rows as in TileArgs (level k at row 2 + k), else NULL
    int32_t m;
    double vscale;
};

template <typename real>
__global__ void __launch_bounds__(kSmallThreadsGrad) small_grad_kernel(const __grid_constant__ SmallGradJob j) {
    using C2 = typename C2T<real>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = j.n;
    const uint32_t dim = 1u << n;
    C2* ps = reinterpret_cast<C2*>(smem_raw);
    C2* lm = ps + dim;
    __shared__ uint64_t gm[kMaxN];
    __shared__ double sred[kSmallThreadsGrad / 32];
    using WA = typename WAcc<real>::type;
    using SWA = typename WAcc<real>::stype;
    const WA* W = reinterpret_cast<const WA*>(j.wfix);
    // C(z): the cut count, or the weighted sum of the value row
    auto cval = [&](uint32_t z) -> double {
        return W ? (double)(SWA)wsum_full(W, j.m, 1, z) * j.vscale : (double)cut_count_full(gm, n, z);
    };
    const uint32_t tid = threadIdx.x;
    if (tid < (uint32_t)n) gm[tid] = j.gmask[tid];
    __syncthreads();
    const C2* src = reinterpret_cast<const C2*>(j.state);
    for (uint32_t z = tid; z < dim; z += kSmallThreadsGrad) {
        const C2 q = src[z];
        const real cc = (real)cval(z);
        ps[z] = q;
        lm[z] = make_c2(cc * q.x, cc * q.y);
    }
    auto block_sum = [&](double v) -> double {
        v = warp_sum_double(v);
        __syncthreads();
        if ((tid & 31u) == 0) sred[tid >> 5] = v;
        __syncthreads();
        double r = 0.0;
        for (int w = 0; w < kSmallThreadsGrad / 32; ++w) r += sred[w];
        return r;
    };
    const C2* mix = reinterpret_cast<const C2*>(j.mix);
    for (int k = j.levels - 1; k >= 0; --k) {
        __syncthreads();
        double pb = 0.0;
        for (int q = 0; q < n; ++q)
            for (uint32_t i = tid; i < dim / 2; i += kSmallThreadsGrad) {
                const uint32_t lo = i & ((1u << q) - 1u);
                const uint32_t za = ((i >> q) << (q + 1)) | lo, zb = za | (1u << q);
                const C2 a = ps[za], b = ps[zb], la = lm[za], lb = lm[zb];
                pb += (double)((la.x * b.y - la.y * b.x) + (lb.x * a.y - lb.y * a.x));
            }
        const double sb = block_sum(pb);
        if (tid == 0) j.acc[k] = sb;
        const C2 cs = mix[3 * k];
        for (int q = 0; q < n; ++q) {
            __syncthreads();
            for (uint32_t i = tid; i < dim / 2; i += kSmallThreadsGrad) {
                const uint32_t lo = i & ((1u << q) - 1u);
                const uint32_t za = ((i >> q) << (q + 1)) | lo, zb = za | (1u << q);
                rx_pair(ps[za], ps[zb], cs.x, -cs.y);
                rx_pair(lm[za], lm[zb], cs.x, -cs.y);
            }
        }
        __syncthreads();
        double pg = 0.0;
        for (uint32_t z = tid; z < dim; z += kSmallThreadsGrad) {
            const C2 p = ps[z], l = lm[z];
            pg += cval(z) * (double)(l.x * p.y - l.y * p.x);
        }
        const double sg = block_sum(pg);
        if (tid == 0) j.acc[j.levels + k] = sg;
        if (k > 0) {
            const C2* Tk = reinterpret_cast<const C2*>(j.phase) + (size_t)k * j.E1;
            for (uint32_t z = tid; z < dim; z += kSmallThreadsGrad) {
                const C2 f = W ? phase_tab(wsum_full(W, j.m, 2 + k, z), Tk) : Tk[cut_count_full(gm, n, z)];
                const C2 fc = make_c2(f.x, -f.y);
                ps[z] = cmul(ps[z], fc);
                lm[z] = cmul(lm[z], fc);
            }
        }
    }
}

// ---------------------------------------------------------------------------------- small states

constexpr int kSmallThreads = 512;

template <typename real>
__device__ __forceinline__ void small_body(const SmallJob& j) {
    using C2 = typename C2T<real>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* st = reinterpret_cast<C2*>(smem_raw);
    __shared__ uint64_t gm[kMaxN];
    __shared__ double sred[2][kSmallThreads / 32];
    using WA = typename WAcc<real>::type;
    using SWA = typename WAcc<real>::stype;
    const WA* W = reinterpret_cast<const WA*>(j.wfix);  // NULL: unit weights
    const int n = j.n;
    const uint32_t dim = 1u << n;
    const uint32_t tid = threadIdx.x;
    if (tid < (uint32_t)n) gm[tid] = j.gmask[tid];
    C2* gstate = reinterpret_cast<C2*>(j.state);
    for (uint32_t z = tid; z < dim; z += kSmallThreads)
        st[z] = j.synth ? make_c2((real)j.init_amp, (real)0) : gstate[z];
    __syncthreads();

    const C2* mix = reinterpret_cast<const C2*>(j.mix);
    for (int k = 0; k < j.levels; ++k) {
        const C2* T = reinterpret_cast<const C2*>(j.phase) + (size_t)k * j.E1;
        if (W)
            for (uint32_t z = tid; z < dim; z += kSmallThreads) st[z] = cmul(st[z], phase_tab(wsum_full(W, j.m, 2 + k, z), T));
        else
            for (uint32_t z = tid; z < dim; z += kSmallThreads) st[z] = cmul(st[z], __ldg(T + cut_count_full(gm, n, z)));
        const C2 cs = mix[3 * k];
        for (int q = 0; q < n; ++q) {
            __syncthreads();
            for (uint32_t i = tid; i < dim / 2; i += kSmallThreads) {
                const uint32_t lo = i & ((1u << q) - 1u);
                const uint32_t za = ((i >> q) << (q + 1)) | lo;
                rx_pair(st[za], st[za | (1u << q)], cs.x, cs.y);
            }
        }
        __syncthreads();
    }

    if (j.cutval) {
        if (W)
            for (uint32_t z = tid; z < dim; z += kSmallThreads) j.cutout_w[z] = (double)(SWA)wsum_full(W, j.m, 1, z) * j.vscale;
        else
            for (uint32_t z = tid; z < dim; z += kSmallThreads) j.cutout[z] = (uint16_t)cut_count_full(gm, n, z);
    }

    if (j.expect) {
        double sc = 0.0, sn = 0.0;
        for (uint32_t z = tid; z < dim; z += kSmallThreads) {
            const double p = (double)st[z].x * (double)st[z].x + (double)st[z].y * (double)st[z].y;
            sn += p;
            sc += p * (W ? (double)(SWA)wsum_full(W, j.m, 1, z) * j.vscale : (double)cut_count_full(gm, n, z));
        }
        sc = warp_sum_double(sc);
        sn = warp_sum_double(sn);
        if ((tid & 31u) == 0) {
            sred[0][tid >> 5] = sc;
            sred[1][tid >> 5] = sn;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < kSmallThreads / 32; ++w) {
                a += sred[0][w];
                b += sred[1][w];
            }
            j.partials[0] = make_double2(a, b);
        }
    }
    if (j.store)
        for (uint32_t z = tid; z < dim; z += kSmallThreads) gstate[z] = st[z];
}

template <typename real>
__global__ void __launch_bounds__(kSmallThreads) small_kernel(const __grid_constant__ SmallJob j) {
    small_body<real>(j);
}

template <typename real>
__global__ void __launch_bounds__(kSmallThreads) small_batch_kernel(const SmallJob* __restrict__ jobs) {
    small_body<real>(jobs[blockIdx.x]);
}

// ---------------------------------------------------------------------------------- coefficients

// Per level k: T_k[c] = exp(-i gamma_k c) for c = 0..|E| (the last level's table times the
// exact factor g = gre + i gim), and the mixer entries (cos b, sin b), (t, 0), (f, 0) with
// RX(2b) = f [[1, -it], [-it, 1]] (fold = 0: t = tan b, f = cos b) or
// RX(2b - pi) = f [[1, -it], [-it, 1]] (fold = 1: t = -cot b, f = sin b).
// With fold_factors, the tile passes never multiply by f: the n factors of level k-1's mixer are
// folded into T_k, and those of the chunk's last mixer into the last table as well (real
// scalars commute with every gate; between two phases the state is off by at most
// (1 / |f|)^n <= 2^(n/2), far inside the floating-point range).
// The butterflies use t rounded to the state precision (t~), so f is taken as
// sign(cos b or sin b) / sqrt(1 + t~^2): each butterfly is then an exact rotation (by atan t~,
// within half an ulp of t from the requested angle) and the level keeps the norm up to the
// arithmetic rounding, instead of drifting by f^2 (1 + t~^2) per qubit.
template <typename real>
__device__ __forceinline__ double mixer_factor(double beta, int fold) {
    double s, co;
    sincos(beta, &s, &co);
    const double tr = (double)(real)(fold ? -co / s : s / co);  // the coefficient the passes use
    return copysign(1.0 / sqrt(1.0 + tr * tr), fold ? s : co);
}

// Fixed-point rows of an edge-weighted graph (see the weighted split above).  Row 0: endpoints;
// row 1: value weights round(w_e 2^S) as signed B-bit words; row wrow0 + k: level k's angles
// gamma_k w_e / (2 pi) modulo one turn, in units of 2^-B turns.  All in FP64 before rounding.
template <typename real>
__device__ void coeff_weighted_rows(const CoeffArgs& a, int k) {
    using WA = typename WAcc<real>::type;
    using SWA = typename WAcc<real>::stype;
    constexpr double kTurn = sizeof(WA) == 4 ? 4294967296.0 : 18446744073709551616.0;
    WA* W = reinterpret_cast<WA*>(a.wfix);
    const double inv2pi = 0.15915494309189533577;  // 1 / (2 pi)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.m; e += gridDim.x * blockDim.x) {
        if (k == 0) {
            W[e] = (WA)a.uv[e];
            W[a.m + e] = (WA)(SWA)llrint(a.w[e] * a.vmul);
        }
        if (k < a.levels) {
            double t = a.gamma[k] * a.w[e] * inv2pi;
            t -= floor(t);                      // [0, 1) turns, exact
            double u = rint(t * kTurn);         // t * 2^B has at most 53 significant bits
            if (u >= kTurn) u = 0.0;            // one full turn
            W[(size_t)(a.wrow0 + k) * a.m + e] = (WA)(unsigned long long)u;
        }
    }
}

template <typename real>
__device__ __forceinline__ void coeff_body(const CoeffArgs& a, const int k) {
    using C2 = typename C2T<real>::type;
    C2* T = reinterpret_cast<C2*>(a.phase) + (size_t)k * a.E1;
    const bool last = k == a.levels - 1;
    double mult = 1.0;
    if (a.fold_factors) {
        if (k > 0) mult *= pow(mixer_factor<real>(a.beta[k - 1], a.fold[k - 1]), (double)a.n);
        if (last) mult *= pow(mixer_factor<real>(a.beta[k], a.fold[k]), (double)a.n);
    }
    if (a.sweep && k < a.levels) {
        const double f = mixer_factor<real>(a.beta[k], a.fold[k]);
        mult = pow(fabs(f), (double)a.n);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double q = 1.0;
            for (int sdone = 0; sdone <= kMaxN; ++sdone, q *= f * f) a.gpow[(size_t)k * (kMaxN + 1) + sdone] = q;
        }
    }
    if (a.weighted) coeff_weighted_rows<real>(a, k);
    if (k >= a.levels) return;  // levels == 0: only the endpoint and value rows
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.E1; c += gridDim.x * blockDim.x) {
        double s, co;
        if (a.weighted)  // rotation steps of a turn (the weighted sums carry gamma_k)
            sincospi((double)c * (2.0 / kWTurnSteps), &s, &co);
        else
            sincos(a.gamma[k] * (double)c, &s, &co);
        double re = co * mult, im = -s * mult;
        if (last) {  // (re + i im)(gre + i gim), exact for g in {1, -i, -1, i}
            const double r2 = re * a.gre - im * a.gim, i2 = re * a.gim + im * a.gre;
            re = r2;
            im = i2;
        }
        T[c] = make_c2((real)re, (real)im);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s, co;
        sincos(a.beta[k], &s, &co);
        C2* m = reinterpret_cast<C2*>(a.mix) + 3 * k;
        m[0] = make_c2((real)co, (real)s);
        if (!a.fold[k]) {
            m[1] = make_c2((real)(s / co), (real)0);
            m[2] = make_c2((real)co, (real)0);
        } else {
            m[1] = make_c2((real)(-co / s), (real)0);
            m[2] = make_c2((real)s, (real)0);
        }
    }
}

template <typename real>
__global__ void coeff_kernel(const __grid_constant__ CoeffArgs a) {
    coeff_body<real>(a, blockIdx.y);
}

// The coefficients of several requests in one launch (the server's packed mid-size states):
// blockIdx.z picks the request, whose CoeffArgs are read from the device array.
template <typename real>
__global__ void coeff_batch_args_kernel(const CoeffArgs* __restrict__ args) {
    coeff_body<real>(args[blockIdx.z], blockIdx.y);
}

// Batched coefficient tables for packed small states: CTA b builds job b's plain per-level
// phase tables and (cos b, sin b) mixer entries (no folded factors; small states use plain RX).
struct CoeffJob {
    int32_t levels, E1;
    const double* gamma;
    const double* beta;
    void* phase;  // [level][E1]
    void* mix;    // [3 * level]
};

template <typename real>
__global__ void coeff_batch_kernel(const CoeffJob* __restrict__ jobs) {
    using C2 = typename C2T<real>::type;
    const CoeffJob j = jobs[blockIdx.x];
    for (int k = 0; k < j.levels; ++k) {
        C2* T = reinterpret_cast<C2*>(j.phase) + (size_t)k * j.E1;
        for (int c = threadIdx.x; c < j.E1; c += blockDim.x) {
            double s, co;
            sincos(j.gamma[k] * (double)c, &s, &co);
            T[c] = make_c2((real)co, (real)(-s));
        }
        if (threadIdx.x == 0) {
            double s, co;
            sincos(j.beta[k], &s, &co);
            C2* m = reinterpret_cast<C2*>(j.mix) + 3 * k;
            m[0] = make_c2((real)co, (real)s);
            m[1] = make_c2((real)0, (real)0);
            m[2] = make_c2((real)1, (real)0);
        }
    }
}

// Resolves the pending transforms of a state in place, one index pair (i, dim - 1 - i) per
// step: with `parity`, the (re, im) halves of every amplitude at an odd-parity index are swapped
// (the parity form of the forward passes; the swap is its own inverse, so the same kernel also
// enters the form); with `complement`, psi_z <-> psi_{~z}.
template <typename real>
__global__ void complement_kernel(void* state, uint64_t dim, int complement, int parity) {
    using C2 = typename C2T<real>::type;
    C2* s = reinterpret_cast<C2*>(state);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim / 2; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = dim - 1 - i;
        C2 a = s[i], b = s[j];
        if (parity) {
            if (__popcll(i) & 1) a = make_c2(a.y, a.x);
            if (__popcll(j) & 1) b = make_c2(b.y, b.x);
        }
        if (complement) {
            s[i] = b;
            s[j] = a;
        } else {
            s[i] = a;
            s[j] = b;
        }
    }
}

// ---------------------------------------------------------------------------------- reductions / fill

__device__ __forceinline__ void finalize_body(const double2* __restrict__ partials, uint64_t count,
                                              double2* __restrict__ out) {
    __shared__ double sc[1024], sn[1024];
    double a = 0.0, b = 0.0;
    for (uint64_t i = threadIdx.x; i < count; i += 1024) {
        const double2 p = partials[i];
        a += p.x;
        b += p.y;
    }
    sc[threadIdx.x] = a;
    sn[threadIdx.x] = b;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sc[threadIdx.x] += sc[threadIdx.x + s];
            sn[threadIdx.x] += sn[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = make_double2(sc[0], sn[0]);
}

static __global__ void __launch_bounds__(1024) finalize_kernel(const double2* __restrict__ partials, uint64_t count,
                                                        double2* __restrict__ out) {
    finalize_body(partials, count, out);
}

// finalize_kernel for blockIdx.x of several requests whose partials lie back to back, `count`
// each (the same summation order, so each result equals the lone reduction bit for bit).
static __global__ void __launch_bounds__(1024) finalize_batch_kernel(const double2* __restrict__ partials,
                                                              uint64_t count, double2* __restrict__ out) {
    finalize_body(partials + (size_t)blockIdx.x * count, count, out + blockIdx.x);
}

template <typename real>
__global__ void fill_kernel(void* state, uint64_t dim, double amp) {
    using C2 = typename C2T<real>::type;
    C2* s = reinterpret_cast<C2*>(state);
    const C2 val = make_c2((real)amp, (real)0);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (uint64_t)gridDim.x * blockDim.x)
        s[i] = val;
}

}  // namespace qaoa
