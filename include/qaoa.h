/*
 * qaoa.h -- C ABI of the B300 QAOA max-cut state-vector simulator.
 *
 * The library simulates the QAOA circuit of the paper's Algorithm 1 (Section 2.1) for the
 * max-cut problem, using the paper's rotation compression (Eqs. rewrite_UC .. UC_opt,
 * Algorithm 2), launch control (Section 2.2) and the popcount cut count of Algorithm 3
 * (Section 2.3), on one GPU with hand-written sm_103a kernels.
 *
 * Conventions (fixed here because the paper's own definition of the cost Hamiltonian is not
 * part of its text):
 *   - qubit u is bit u of the basis index z (least significant bit = qubit 0);
 *   - C(z) = sum over edges (u, v) of w_uv * (bit u of z XOR bit v of z);
 *   - the initial state is |+>^n, every amplitude 2^(-n/2) (launch control, Section 2.2);
 *   - level k applies psi_z <- exp(-i gamma_k C(z)) psi_z, then RX(2 beta_k) =
 *     [[cos beta_k, -i sin beta_k], [-i sin beta_k, cos beta_k]] on every qubit.
 *     The paper's gamma is minus this gamma and its RX angle is 2 beta (global phase aside);
 *   - <C> = sum_z |psi_z|^2 C(z).
 *
 * Memory: a state of 2^n amplitudes lives in a device buffer the CALLER allocates and owns
 * (complex64 = 2 x float32 interleaved, complex128 = 2 x float64 interleaved, index z).  The
 * library borrows it; it takes only small workspace of its own (phase tables, per-tile
 * partial sums) at qaoa_state_init and gives it back at qaoa_state_free.  That workspace comes
 * from a stream-ordered memory pool the library keeps per device (cudaMallocFromPoolAsync on the
 * state's stream), which holds on to up to 256 MiB of freed blocks for later states, so creating
 * and freeing states in a loop costs no cudaMalloc or cudaFree once the pool is warm.  Host
 * arrays passed in are copied before the call returns; the caller may free them afterwards.
 *
 * Errors: every entry point returns a qaoa_status; negative values are errors and
 * qaoa_last_error() returns a message for the calling thread.  Nothing aborts and no C++
 * exception crosses the ABI.  Work is enqueued on the CUDA stream given at init; calls that
 * return host results synchronise that stream.
 *
 * Threads: distinct state handles may be used from different host threads at the same time
 * (each with its own stream); one handle must not be used by two threads at once.
 */
#ifndef QAOA_B300_QAOA_H
#define QAOA_B300_QAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QAOA_OK = 0,
    QAOA_PENDING = 1,           /* serving: result not ready yet */
    QAOA_ERR_INVALID = -1,      /* bad argument (graph, size, angle, handle) */
    QAOA_ERR_OOM = -2,          /* workspace allocation failed */
    QAOA_ERR_CUDA = -3,         /* a CUDA call failed; message in qaoa_last_error() */
    QAOA_ERR_AGAIN = -4,        /* serving: queue full, retry later */
    QAOA_ERR_TIMEOUT = -5,      /* serving: deadline passed */
    QAOA_ERR_UNSUPPORTED = -6   /* valid request this build cannot run */
} qaoa_status;

typedef enum { QAOA_C64 = 0, QAOA_C128 = 1 } qaoa_prec;

/* Problem statement of Table 1 (Section 2.1): N vertices (= qubits), the edge list that the
 * upper-triangular matrix `graph` encodes, and optional edge weights `w`.
 *   n       : 1 <= n <= 34
 *   m       : number of edges, m >= 0
 *   edges   : 2*m int32 endpoints (u0, v0, u1, v1, ...), 0 <= u, v < n, u != v, no pair twice
 *   weights : NULL for unit weights (Algorithm 3); otherwise m finite doubles w_e with
 *             |w_e| <= 1e12 (Algorithm 2: C(z) = sum_e w_e (z_u xor z_v)); negative weights
 *             are allowed.  Weights that are all exactly 1 take the unit-weight path.
 * With weights, the kernels evaluate two sums per amplitude in B-bit fixed point (B = 32 for
 * complex64, 64 for complex128), each exact modulo 2^B: the phase angle gamma_k C(z) from
 * per-edge angles gamma_k w_e / (2 pi) rounded to 2^-B turns (error at most m 2^-B turns), and
 * the value C(z) from weights rounded to 2^-S with S the largest power such that
 * sum |w_e| 2^S <= 2^(B-2) (error at most m 2^-(S+1)). */
typedef struct {
    int32_t n;
    int32_t m;
    const int32_t *edges;
    const double *weights;
} qaoa_graph;

typedef struct qaoa_state_s *qaoa_state; /* opaque; owned by the library */

/* Bytes a state of n qubits needs: 2^n * 8 (complex64) or 2^n * 16 (complex128); 0 if n is
 * out of range. */
size_t qaoa_state_bytes(int32_t n, qaoa_prec prec);

/* Binds a caller-owned device buffer (at least qaoa_state_bytes(n, prec) bytes, 16-byte
 * aligned) and a CUDA stream (cudaStream_t passed as void*, NULL = legacy default stream) to a
 * new state handle holding |+>^n (Section 2.2, launch control).  The buffer is not written
 * here: the uniform amplitudes are produced by the first kernel that needs them, so the first
 * level of qaoa_apply_layers reads nothing.  Validates the graph (QAOA_ERR_INVALID on a self
 * loop, repeated edge, endpoint out of range, non-finite weight or |w| > 1e12), encodes the
 * rows graph_I of Table 1 and the pass plan, and takes its workspace from the library's pool on
 * that stream (QAOA_ERR_OOM).  The buffer and the stream must stay valid until qaoa_state_free
 * returns.  On success *out receives the handle. */
qaoa_status qaoa_state_init(const qaoa_graph *g, qaoa_prec prec, void *dev_buf, size_t buf_bytes,
                            void *cuda_stream, qaoa_state *out);

/* Returns the state to |+>^n (deferred, nothing is written) keeping the graph, buffer, stream
 * and workspace: the initial layer of Algorithm 1 by launch control (Section 2.2). */
qaoa_status qaoa_state_reset(qaoa_state s);

/* Makes the caller's buffer hold psi_z at index z: writes out a still-deferred |+>^n and
 * resolves a pending index complement.  (When |tan beta_k| > 1 the tile passes evaluate
 * RX(2 beta) as -i X RX(2 beta - pi) with X on every qubit; X maps index z to ~z and commutes with
 * the cost phase and the mixer, so the library records it instead of moving data, and <C> is
 * unaffected.)  Stream-ordered, no host synchronisation.  qaoa_state_copy_out does this itself;
 * call it before reading the buffer directly. */
qaoa_status qaoa_state_sync(qaoa_state s);

/* Applies p levels (Algorithm 1's level loop) with angles gamma[0..p-1], beta[0..p-1] on top
 * of the current state: per level, the rotation-compressed cost phase (Eq. UC_opt with the
 * popcount count of Algorithm 3, evaluated on the fly) and the RX mixer on every qubit.
 * Asynchronous on the state's stream; the angle arrays are copied before return.  p == 0
 * does what qaoa_state_sync does.  QAOA_ERR_INVALID on p < 0 or non-finite angles.  Until
 * qaoa_state_sync, the buffer may hold the state with its indices complemented (see there). */
qaoa_status qaoa_apply_layers(qaoa_state s, int32_t p, const double *gamma, const double *beta);

/* <C> = sum_z |psi_z|^2 C(z) and the squared norm sum_z |psi_z|^2 of the current state,
 * reduced in FP64 in a fixed order (run-to-run identical).  Synchronises the stream. */
qaoa_status qaoa_expectation(qaoa_state s, double *out_c, double *out_norm);

/* <C> of the p-level circuit from |+>^n and its gradient d<C>/d gamma_k, d<C>/d beta_k
 * (k = 0..p-1), by one forward run and one adjoint sweep (no per-level storage).  With
 * psi_k the state after level k and lambda_k = (U_p .. U_{k+1})^dagger C psi_p:
 *   d<C>/d beta_k  = 2 Im <lambda_k| sum_j X_j |psi_k>,
 *   d<C>/d gamma_k = 2 Im <M_k^dagger lambda_k| C |M_k^dagger psi_k>,
 * and psi, lambda are uncomputed level by level with the inverse mixer and phase.  The sweep
 * keeps psi in the state buffer and lambda in dev_work, a caller-owned device buffer of at
 * least qaoa_state_bytes(n, prec) bytes (16-byte aligned, not the state buffer), which it
 * overwrites.  Sums are reduced in FP64 in a fixed order.  Afterwards the state is |+>^n
 * (deferred).  Writes <C> to *out_c (may be NULL) and the 2p derivatives to d_gamma[0..p-1] and
 * d_beta[0..p-1]; synchronises the stream.  Takes gradient workspace from the library's pool on
 * first use (p phase tables, 2 doubles per tile), kept until qaoa_state_free.  QAOA_ERR_INVALID
 * on p < 1, non-finite angles or a bad buffer; QAOA_ERR_OOM if the workspace cannot be had. */
qaoa_status qaoa_gradient(qaoa_state s, int32_t p, const double *gamma, const double *beta,
                          void *dev_work, size_t work_bytes, double *out_c, double *d_gamma,
                          double *d_beta);

/* Copies the current state (bytes = qaoa_state_bytes) to host memory, writing out a deferred
 * |+>^n first.  Synchronises the stream.  Parity hook. */
qaoa_status qaoa_state_copy_out(qaoa_state s, void *host_dst, size_t bytes);

/* Gives the handle's workspace back to the library's pool (stream-ordered, on the state's
 * stream), waits for the stream's pending work and releases the handle; never frees the
 * caller's buffer.  NULL is accepted. */
qaoa_status qaoa_state_free(qaoa_state s);

/* Cut value C(z) of every basis state (Algorithm 3 on the GPU, computed by the same device
 * code the cost phase uses), written to host_out[0 .. 2^n - 1].  Unit weights only
 * (QAOA_ERR_INVALID for a weighted graph); n <= 30.  Runs on the current device's legacy
 * default stream and synchronises it.  Parity hook. */
qaoa_status qaoa_cut_table(const qaoa_graph *g, uint16_t *host_out);

/* C(z) of every basis state as doubles, for unit or edge-weighted graphs (Algorithm 2's cut
 * value, from the same device code as <C> and the adjoint's C psi), evaluated in precision
 * prec's fixed point (see qaoa_graph) under the geometry of mixer group `group` and register
 * layout `layout` (group < 0: the path the state size uses by default).  n <= 28.  Synchronous,
 * legacy default stream.  Parity hook. */
qaoa_status qaoa_cut_table_f64(const qaoa_graph *g, qaoa_prec prec, int32_t group, int32_t layout,
                               double *host_out);

/* Same as qaoa_cut_table, but evaluated under the tile geometry of mixer group `group`
 * (0 = the low group) of the pass plan for precision `prec`, in register layout `layout`
 * (0, 1 or 2).  Lets tests check every split of the cut count the kernels use.  Parity
 * hook; QAOA_ERR_INVALID for a group or layout the plan does not have. */
qaoa_status qaoa_cut_table_geometry(const qaoa_graph *g, qaoa_prec prec, int32_t group,
                                    int32_t layout, uint16_t *host_out);

/* Host-only description of the pass plan for n qubits, precision prec and p levels (no GPU
 * needed).  Writes up to cap int32 values into out and returns the number needed in *count:
 *   [Q, R, c_min, n_groups, (size, bit indices...) per group, n_passes,
 *    per pass: (group, n_ops, (kind, arg, mask) per op)]
 * kind: 1 load, 2 synthesise |+> (arg = layout), 3 exchange (arg = layout), 4 RX (arg =
 * level, mask = local target bits), 5 phase (arg = level), 6 expectation, 7 store, 8 cut
 * values; the adjoint sweep's plan (not described here) also uses 9 lambda = C psi, 10 inverse
 * RX with pair sums, 11 gamma sums and 12 conjugate phase (arg = level | slot << 16).  Small
 * states (whole state in one CTA) have no pass plan: *count = 0.  For tests of the
 * planner: every level must apply RX to every qubit exactly once, phases in order. */
qaoa_status qaoa_plan_describe(int32_t n, qaoa_prec prec, int32_t p, int32_t *out, int32_t cap,
                               int32_t *count);

/* Launch statistics, for the benchmark's roofline.  When enabled, every state-pass kernel
 * launch is bracketed by CUDA events on the state's stream. */
typedef struct {
    int64_t kernel_launches;     /* all kernels this handle launched since the last reset */
    int64_t pass_launches;       /* read+write state passes among them */
    double pass_ms;              /* summed event time of those passes */
    double pass_bytes;           /* algorithmic bytes of those passes: 2 * 2^n * element size each */
    int64_t synth_launches;      /* passes that write without reading (deferred |+>^n) */
    double synth_ms;
    double synth_bytes;
    /* the read+write passes split by program: [0] mixer only, [1] with the cost phase (the
     * fused boundary passes), [2] with <C> (the last pass) */
    int64_t kind_launches[3];
    double kind_ms[3];
} qaoa_profile_stats;

/* Index checks (a development aid; the paper has no counterpart).  A library built with
 * -DQAOA_DEBUG_BOUNDS (`python -m paper_2312_03019_b300.build --debug-bounds`, written to
 * libqaoa_b300_debug.so) checks, in its pass and adjoint kernels, every state load and store,
 * shared-memory exchange, phase-table read, cut-value write and weighted-row read against the
 * buffer it belongs to; a failed check sets a bit in one word on the device and skips the access
 * (1 state load, 2 state store, 4 shared-memory write, 8 shared-memory read, 16 phase-table
 * read, 32 cut-value write, 64 weighted row read).  This call synchronises `device`, returns the
 * word in *out_flags (0: no check failed since it was last cleared) and clears it if `clear`.
 * A release build returns QAOA_ERR_UNSUPPORTED. */
qaoa_status qaoa_debug_bounds_read(int32_t device, uint32_t *out_flags, int32_t clear);

/* enable != 0 starts recording (and resets the counters); 0 stops. */
qaoa_status qaoa_profile_enable(qaoa_state s, int32_t enable);
/* Synchronises the stream and returns the counters since the last enable. */
qaoa_status qaoa_profile_read(qaoa_state s, qaoa_profile_stats *out);

/* <C> and the squared norm of a complex64 / complex128 state that the caller already holds on the
 * device, computed without allocating anything.  The paper has no counterpart: this entry
 * exists for callers that cannot call cudaMalloc -- for example a runtime that has handed all
 * of the GPU's memory to its own pool, or a loop that must not pay the device-wide
 * synchronisation an allocation can cause.  It takes the graph (as for qaoa_state_init), the
 * state (2^n amplitudes at dev_state, state_bytes >= qaoa_state_bytes(n, prec), 16-byte
 * aligned, read only) and a CUDA stream (NULL = legacy default stream), and returns both sums
 * through the host pointers, synchronising the stream.
 *
 * Scratch space is a fixed 1 MiB array in the library's device memory (one partial pair per
 * tile of the state plus the result), which every GPU that loads the library keeps until the
 * process exits.  That bounds the size: n <= 29 for complex64 and n <= 28 for complex128
 * (larger n returns QAOA_ERR_INVALID with a message).  Each call looks up the array's address on
 * the current device (cudaGetSymbolAddress, no allocation), so the call is right after a
 * cudaDeviceReset too.  All calls share the one array: every entry a call reads is written
 * earlier in the same call, so nothing has to be cleared, but two calls whose work overlaps on
 * the GPU (on different streams or host threads) race on it and give wrong results.
 * QAOA_ERR_INVALID as well when dev_state is not device (or managed) memory of the current
 * device -- a host, pinned or other-device pointer is refused before any launch -- and when the
 * stream is being captured into a CUDA graph (the call synchronises the stream).  Unit weights
 * only: a weights array whose entries are all exactly 1 is the unit-weight graph; any other
 * weight returns QAOA_ERR_UNSUPPORTED. */
qaoa_status qaoa_expectation_static(const qaoa_graph *g, qaoa_prec prec, const void *dev_state,
                                    size_t state_bytes, void *cuda_stream, double *out_c,
                                    double *out_norm);

/* ------------------------------------------------------------------------- serving
 * A request loop for QAOA evaluations as a classical optimiser emits them (the paper's Fig. 1
 * workflow; the paper itself describes no server).  A scheduler thread owns the GPU work:
 *   - admission in arrival order, by HBM footprint: each request needs its state (2^n amplitudes)
 *     plus, for gradients, the adjoint buffer and small tables, carved from one device arena of
 *     hbm_budget_bytes allocated at qaoa_server_create; at most max_inflight requests at once;
 *   - continuous batching: every scheduler turn packs all admitted small forward requests (whole
 *     state in one CTA: n <= 14 for complex64, n <= 13 for complex128) into one batched launch,
 *     one CTA per request, and the admitted mid-size complex64 forward requests (15 <= n <= 22,
 *     p <= 8, unit weights) of one (n, p) into packed launches (one launch per pass over every
 *     tile of up to 32 requests), while larger requests run concurrently on a pool of `streams`
 *     CUDA streams; with two or more streams, requests whose state fills the GPU on its own
 *     (64 MiB or more: n >= 23 complex64, n >= 22 complex128) run one after another on stream 0
 *     at the lowest stream priority, and everything else on streams 1.. at the highest, so short
 *     requests overtake the long passes instead of queueing behind them; with use_graphs each
 *     launch sequence is recorded into a CUDA graph and replayed through an executable graph
 *     cached per request shape;
 *   - completion is detected with CUDA events; results land in pinned host memory.
 * Each result is computed by the same kernels and reduction order as a lone request, so it is
 * identical alone and in the mix. */
#define QAOA_SERVE_MAX_P 64

typedef struct {
    size_t hbm_budget_bytes;  /* device arena size for states and per-request workspace */
    int32_t max_inflight;     /* requests on the GPU at once (>= 1) */
    int32_t queue_capacity;   /* queued requests before qaoa_submit returns QAOA_ERR_AGAIN */
    int32_t max_batch;        /* small requests packed per launch (1..256) */
    int32_t streams;          /* CUDA streams for concurrent requests (1..64) */
    int32_t use_graphs;       /* 1: replay captured CUDA graphs; 0: plain launches */
    qaoa_prec prec;           /* precision of every state of this server */
} qaoa_server_config;

typedef struct {
    qaoa_graph graph;     /* copied at submit */
    int32_t p;            /* 1 <= p <= QAOA_SERVE_MAX_P */
    const double *gamma;  /* p angles, copied at submit */
    const double *beta;   /* p angles, copied at submit */
    int32_t want_grad;    /* 1: also d<C>/d gamma, d<C>/d beta (adjoint sweep) */
    double deadline_s;    /* 0: none; else seconds after submit by which the request must have
                           * been dispatched to the GPU: one still queued then completes with
                           * status QAOA_ERR_TIMEOUT without running (work already dispatched
                           * always finishes) */
} qaoa_request;

typedef struct {
    int32_t status;       /* QAOA_OK or the error the request failed with */
    int32_t p;
    int32_t has_grad;
    int32_t batched;      /* 1: ran in a packed small-request launch */
    double expectation;   /* <C> */
    double norm;          /* sum |psi|^2 */
    double t_submit;      /* server clock (qaoa_server_time) at submit */
    double t_start;       /* ... when dispatched to the GPU */
    double t_done;        /* ... when the scheduler saw it complete */
    double d_gamma[QAOA_SERVE_MAX_P];
    double d_beta[QAOA_SERVE_MAX_P];
} qaoa_result;

typedef struct {
    int64_t submitted, completed, failed, rejected_full;
    int64_t batches, batched_requests, single_requests, graph_launches;
    size_t arena_peak_bytes;
    int64_t timed_out;    /* requests whose deadline passed before dispatch (counted in failed) */
    int64_t tiled_batches;          /* packed launches of mid-size (tiled) states */
    int64_t tiled_batched_requests; /* requests that ran in them (also counted in batched_requests) */
} qaoa_server_stats;

typedef struct qaoa_server_s *qaoa_server;

/* Creates the server and starts its scheduler thread on the current device.  Allocates the arena,
 * pinned result buffers, streams and events (QAOA_ERR_OOM if the arena does not fit). */
qaoa_status qaoa_server_create(const qaoa_server_config *cfg, qaoa_server *out);
/* Queues a request (graph and angles are copied); *ticket identifies it.  Edge-weighted graphs
 * are accepted and always run alone (never packed with other small requests).  QAOA_ERR_AGAIN when the
 * queue is full; QAOA_ERR_INVALID for a bad request (including a negative or non-finite
 * deadline); QAOA_ERR_OOM when its footprint exceeds the whole arena.  Thread-safe. */
qaoa_status qaoa_submit(qaoa_server sv, const qaoa_request *r, uint64_t *ticket);
/* Non-blocking: QAOA_PENDING while the request is queued or running; QAOA_OK with *out filled
 * (the ticket is then released); QAOA_ERR_INVALID for an unknown ticket.  Thread-safe. */
qaoa_status qaoa_poll(qaoa_server sv, uint64_t ticket, qaoa_result *out);
/* Seconds on the server's monotonic clock (the time base of qaoa_result). */
double qaoa_server_time(qaoa_server sv);
qaoa_status qaoa_server_stats_read(qaoa_server sv, qaoa_server_stats *out);
/* Stops the scheduler after the requests already admitted finish, frees everything. */
qaoa_status qaoa_server_destroy(qaoa_server sv);

/* Message of the last error on the calling thread ("" if none). */
const char *qaoa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_B300_QAOA_H */
