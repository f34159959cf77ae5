// server.cuh -- continuous-batching request server behind qaoa_server_* (included by capi.cu, so
// it shares the state machinery: forward_async, gradient_async, the small-state kernels).
//
// One scheduler thread issues all GPU work.  Each turn it (1) retires requests whose CUDA event
// has completed, (2) admits queued requests in arrival order while the arena has room for their
// footprint and fewer than max_inflight run, (3) packs every admitted small forward request into
// one launch (coefficient tables for all of them, then one CTA per request), and (4) dispatches
// every other admitted request on a stream of the pool: requests that fill the GPU on their own
// in order on a low-priority lane, the rest on the least loaded high-priority stream.  With use_graphs, each
// dispatch's launch sequence is recorded by stream capture and replayed through an executable
// graph kept per shape (a small pool per shape, since one executable graph cannot run
// concurrently with itself; executables are updated in place with cudaGraphExecUpdate).
#pragma once

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <tuple>
#include <unordered_map>

namespace {

// First-fit sub-allocator over one device allocation (256-byte granules, coalescing frees).
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes

    static size_t round(size_t x) { return (x + 255) & ~(size_t)255; }
    void init(char* b, size_t s) {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
    }
    bool alloc(size_t bytes, size_t& off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round(bytes);
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct SReq {
    uint64_t ticket = 0;
    HostGraph g;
    int p = 0;
    std::vector<double> gamma, beta;
    bool grad = false;
    double t_submit = 0.0;
    double deadline = 0.0;  // server clock by which it must be dispatched (0: none)
};

// Device block of a request that runs alone (offsets from the block start).
struct Layout {
    size_t state, work, phase, mix, partials, result, gtab, gmix, gacc, gpart, gpow, wfix, gwfix, total;
};

Layout single_layout(const HostGraph& g, int p, int prec, bool grad, uint64_t ntiles) {
    const int n = g.n;
    const size_t eb = elem_bytes(prec), E1 = (size_t)table_entries(g), dim = (size_t)1 << n;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += Arena::round(bytes);
        return at;
    };
    L.state = take(dim * eb);
    L.work = grad ? take(dim * eb) : 0;
    L.phase = take((size_t)p * E1 * eb);
    L.mix = take((size_t)3 * p * eb);
    L.partials = take(ntiles * sizeof(double2));
    L.result = take(sizeof(double2));
    if (g.weighted) L.wfix = take(wfix_bytes(g, prec, p));
    if (grad) {
        L.gtab = take((size_t)p * E1 * eb);
        L.gmix = take((size_t)3 * p * eb);
        L.gacc = take(grad_acc_bytes(p));
        L.gpart = take(grad_partials_bytes(n, p));
        L.gpow = take((size_t)p * (kMaxN + 1) * sizeof(double));
        if (g.weighted) L.gwfix = take(wfix_bytes(g, prec, p));
    }
    L.total = o;
    return L;
}

// Arena bytes of one packed small forward request: its phase tables and mixer entries.
size_t small_bytes(int m, int p, int prec) {
    const size_t eb = elem_bytes(prec);
    return Arena::round((size_t)p * (m + 1) * eb) + Arena::round((size_t)3 * p * eb);
}

// Packed launch head block (device) and staging slot (pinned host), same layout:
// [CoeffJob x maxB][SmallJob x maxB][angles: maxB x 2 x QAOA_SERVE_MAX_P doubles][results x maxB]
struct BatchLayout {
    size_t coeff, small, angles, results, upload, total;
};

BatchLayout batch_layout(int maxB) {
    BatchLayout L{};
    L.coeff = 0;
    L.small = Arena::round((size_t)maxB * sizeof(CoeffJob));
    L.angles = L.small + Arena::round((size_t)maxB * sizeof(SmallJob));
    L.results = L.angles + Arena::round((size_t)maxB * 2 * QAOA_SERVE_MAX_P * sizeof(double));
    L.upload = L.results;  // bytes copied host -> device per launch
    L.total = L.results + Arena::round((size_t)maxB * sizeof(double2));
    return L;
}

// Packed mid-size forward requests (tiled complex64 states that fit in two mixer groups): one
// launch per pass covers every tile of up to kMidMaxB requests of one (n, p).
constexpr int kMidMaxN = 22;
constexpr int kMidMaxP = 8;
constexpr int kMidMaxB = 32;
constexpr int kMidStages = 4;

// Head block of a packed mid-size launch (device) and its staging slot (pinned host), same layout:
// [TileArgs, pass-major: pass i of request b at i * B + b][CoeffArgs x B][partials: B x tiles]
// [results x B]; the first `upload` bytes go host -> device, the results come back.
struct MidLayout {
    size_t targs, cargs, partials, results, upload, total;
};

MidLayout mid_layout(int passes, int B, uint64_t tiles) {
    MidLayout L{};
    L.targs = 0;
    L.cargs = Arena::round((size_t)passes * B * sizeof(TileArgs<PrecTraits<float>::Q>));
    L.upload = L.cargs + Arena::round((size_t)B * sizeof(CoeffArgs));
    L.partials = L.upload;
    L.results = L.partials + Arena::round((size_t)B * tiles * sizeof(double2));
    L.total = L.results + Arena::round((size_t)B * sizeof(double2));
    return L;
}

// Pinned staging bytes per slot: descriptors of the largest packed launch, and its results.
size_t mid_stage_bytes() {
    const MidLayout L = mid_layout(kMidMaxP + 1, kMidMaxB, 1);
    return L.upload + Arena::round((size_t)kMidMaxB * sizeof(double2));
}

struct Running {  // a request dispatched alone
    SReq r;
    size_t off = 0, bytes = 0;
    qaoa_state_s* st = nullptr;
    int stream = 0, slot = -1;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;  // pooled graph in use (released at completion)
    double t_start = 0.0;
};

struct RunningBatch {
    std::vector<SReq> reqs;
    std::vector<size_t> offs;
    std::vector<size_t> bytes;   // per request (mid-size packs; small packs use small_bytes)
    std::vector<int> slots;      // per request pinned result slots held (mid-size packs)
    bool mid = false;            // packed mid-size states (else small states, one CTA each)
    size_t res_off = 0;          // mid-size packs: offset of the results in the staging slot
    size_t head_off = 0, head_bytes = 0;
    int stream = 0, staging = -1;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    double t_start = 0.0;
};

struct GraphPool {
    std::vector<std::pair<cudaGraphExec_t, bool>> execs;  // (executable, in flight)
};

}  // namespace

struct qaoa_server_s {
    qaoa_server_config cfg{};
    int dev = 0;
    std::chrono::steady_clock::time_point t0;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_load;
    // pinned result slots for single requests: 2 + 2 * QAOA_SERVE_MAX_P doubles each
    double* pin_single = nullptr;
    std::vector<int> free_single;
    // pinned staging for packed launches: descriptors + angles out, results back
    unsigned char* pin_stage = nullptr;
    size_t stage_bytes = 0;
    std::vector<int> free_stage;
    // pinned staging for packed mid-size launches (kMidStages slots of mid_stage_bytes())
    unsigned char* pin_mid = nullptr;
    std::vector<int> free_mid;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::tuple<int, int, int, int>, GraphPool> graphs;  // (kind, n, p, m) -> executables
    // host-side bookkeeping
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SReq> queue;
    std::set<uint64_t> live;
    std::unordered_map<uint64_t, qaoa_result> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    qaoa_server_stats stats{};
    std::thread thr;
    // scheduler-thread only
    std::deque<SReq> pending;
    std::vector<Running> running;
    std::vector<RunningBatch> batches;
    int inflight = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Counters are written by the scheduler thread and read by qaoa_server_stats_read: under the lock.
void bump(qaoa_server_s* sv, int64_t qaoa_server_stats::*field, int64_t k = 1) {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stats.*field += k;
    sv->stats.arena_peak_bytes = sv->arena.peak;
}

bool serve_small(const qaoa_server_s* sv, const SReq& r) {
    return !r.grad && !r.g.weighted && is_small(r.g.n, sv->cfg.prec);
}

cudaEvent_t take_event(qaoa_server_s* sv) {
    if (!sv->event_pool.empty()) {
        cudaEvent_t e = sv->event_pool.back();
        sv->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// A request whose state is at least kLaneBytes fills the GPU on its own (n >= 23 complex64:
// 1024 tiles per pass); two of them running at once only split the memory bandwidth and evict
// each other's state from L2.  With two or more streams, such requests run one after another on
// stream 0, the low-priority lane, and every other request and pack goes to the least loaded of
// the high-priority streams 1.., whose CTAs the block scheduler places ahead of the big passes'.
constexpr uint64_t kLaneBytes = 64ull << 20;

bool fills_gpu(const qaoa_server_s* sv, const SReq& r) {
    return ((1ull << r.g.n) * elem_bytes(sv->cfg.prec)) >= kLaneBytes;
}

int pick_stream(qaoa_server_s* sv, bool big) {
    const int S = (int)sv->streams.size();
    if (S < 2) return 0;
    if (big) return 0;
    int best = 1;
    for (int i = 2; i < S; ++i)
        if (sv->stream_load[i] < sv->stream_load[best]) best = i;
    return best;
}

// Records the work `enqueue` puts on `stream` into a graph and launches it through a pooled
// executable of the same shape (or launches directly when graphs are off).
template <typename F>
qaoa_status run_maybe_graph(qaoa_server_s* sv, std::tuple<int, int, int, int> key, cudaStream_t stream, F&& enqueue,
                            cudaGraphExec_t* used) {
    *used = nullptr;
    if (!sv->cfg.use_graphs) return enqueue();
    CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    qaoa_status st = enqueue();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(stream, &graph);
    if (st != QAOA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    GraphPool& pool = sv->graphs[key];
    cudaGraphExec_t exec = nullptr;
    for (auto& e : pool.execs)
        if (!e.second) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(e.first, graph, &info) == cudaSuccess) {
                exec = e.first;
                e.second = true;
                break;
            }
            cudaGetLastError();
        }
    if (!exec) {
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(ie, "cudaGraphInstantiate");
        }
        pool.execs.push_back({exec, true});
    }
    cudaGraphDestroy(graph);
    CUDA_TRY(cudaGraphLaunch(exec, stream));
    bump(sv, &qaoa_server_stats::graph_launches);
    *used = exec;
    return QAOA_OK;
}

void release_graph(qaoa_server_s* sv, cudaGraphExec_t exec) {
    if (!exec) return;
    for (auto& kv : sv->graphs)
        for (auto& e : kv.second.execs)
            if (e.first == exec) e.second = false;
}

// A state handle over a request's block of the arena (the library's own per-state workspace
// pointers aimed into the block; nothing allocated).
void bind_request_state(qaoa_server_s* sv, qaoa_state_s* st, const SReq& r, char* base, const Layout& L,
                        cudaStream_t stream) {
    st->dev = sv->dev;
    st->n = r.g.n;
    st->prec = sv->cfg.prec;
    st->dim = 1ull << r.g.n;
    st->buf = base + L.state;
    st->stream = stream;
    st->g = r.g;
    st->tc = tile_config_for(sv->cfg.prec);
    st->small = is_small(r.g.n, sv->cfg.prec);
    if (r.g.n > st->tc.Q) {
        st->groups = make_groups(r.g.n, st->tc);
        st->ntiles = 1ull << (r.g.n - st->tc.Q);
    }
    st->d_phase = base + L.phase;
    st->d_mix = base + L.mix;
    st->d_partials = reinterpret_cast<double2*>(base + L.partials);
    st->d_result = reinterpret_cast<double2*>(base + L.result);
    if (r.g.weighted) st->d_wfix = base + L.wfix;
}

// Drops the handle's pointers into the arena (they are not its own) before deleting it.
void unbind_request_state(qaoa_state_s* st) {
    st->d_phase = st->d_mix = nullptr;
    st->d_partials = st->d_result = nullptr;
    st->d_gtab = st->d_gmix = nullptr;
    st->d_gacc = nullptr;
    st->d_gpart = nullptr;
    st->d_gpow = nullptr;
    st->d_wfix = st->d_gwfix = nullptr;
    delete st;
}

template <typename real>
qaoa_status dispatch_single(qaoa_server_s* sv, SReq&& r, size_t off, const Layout& L, int slot) {
    Running run;
    run.off = off;
    run.bytes = L.total;
    run.slot = slot;
    run.stream = pick_stream(sv, fills_gpu(sv, r));
    char* base = sv->arena.base + off;
    qaoa_state_s* st = new (std::nothrow) qaoa_state_s;
    if (!st) return fail(QAOA_ERR_OOM, "host allocation failed");
    bind_request_state(sv, st, r, base, L, sv->streams[run.stream]);
    if (r.grad) {
        st->grad_levels = r.p;
        st->d_gtab = base + L.gtab;
        st->d_gmix = base + L.gmix;
        st->d_gacc = reinterpret_cast<double*>(base + L.gacc);
        st->d_gpart = reinterpret_cast<double2*>(base + L.gpart);
        st->d_gpow = reinterpret_cast<double*>(base + L.gpow);
        if (r.g.weighted) st->d_gwfix = base + L.gwfix;
    }
    run.st = st;
    double* host = sv->pin_single + (size_t)slot * (2 + 2 * QAOA_SERVE_MAX_P);
    void* work = r.grad ? (void*)(base + L.work) : nullptr;
    const int p = r.p;
    auto enqueue = [&]() -> qaoa_status {
        qaoa_status s2 = r.grad ? gradient_async<real>(st, p, r.gamma.data(), r.beta.data(), work)
                                : forward_async<real>(st, p, r.gamma.data(), r.beta.data());
        if (s2 != QAOA_OK) return s2;
        CUDA_TRY(cudaMemcpyAsync(host, st->d_result, sizeof(double2), cudaMemcpyDeviceToHost, st->stream));
        if (r.grad)
            CUDA_TRY(cudaMemcpyAsync(host + 2, st->d_gacc, 2 * (size_t)p * sizeof(double), cudaMemcpyDeviceToHost,
                                     st->stream));
        return QAOA_OK;
    };
    qaoa_status s = run_maybe_graph(sv, std::make_tuple(r.grad ? 2 : 1, r.g.n, p, 0), st->stream, enqueue, &run.exec);
    if (s == QAOA_OK) {
        run.ev = take_event(sv);
        if (!run.ev) s = fail(QAOA_ERR_CUDA, "cudaEventCreate failed");
        else if (cudaEventRecord(run.ev, st->stream) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    }
    if (s != QAOA_OK) {
        release_graph(sv, run.exec);
        if (run.ev) sv->event_pool.push_back(run.ev);
        unbind_request_state(st);
        return s;
    }
    sv->stream_load[run.stream]++;
    run.t_start = sv->now();
    run.r = std::move(r);
    sv->running.push_back(std::move(run));
    bump(sv, &qaoa_server_stats::single_requests);
    return QAOA_OK;
}

// Packed launch of small forward requests: one upload of descriptors and angles, coefficient
// tables for all requests in one launch, then one CTA per request.
template <typename real>
qaoa_status dispatch_batch(qaoa_server_s* sv, std::vector<SReq>&& reqs, std::vector<size_t>&& offs, int staging,
                           size_t head_off) {
    using C2 = typename C2T<real>::type;
    const int B = (int)reqs.size();
    const BatchLayout BL = batch_layout(sv->cfg.max_batch);
    unsigned char* stage = sv->pin_stage + (size_t)staging * sv->stage_bytes;
    char* head = sv->arena.base + head_off;
    CoeffJob* cj = reinterpret_cast<CoeffJob*>(stage + BL.coeff);
    SmallJob* sj = reinterpret_cast<SmallJob*>(stage + BL.small);
    double* ang = reinterpret_cast<double*>(stage + BL.angles);
    double* d_ang = reinterpret_cast<double*>(head + BL.angles);
    double2* d_res = reinterpret_cast<double2*>(head + BL.results);
    double2* res_host = reinterpret_cast<double2*>(stage + BL.results);
    const size_t eb = elem_bytes(sv->cfg.prec);
    int nmax = 1;
    for (int b = 0; b < B; ++b) {
        const SReq& r = reqs[b];
        char* blk = sv->arena.base + offs[b];
        char* phase = blk;
        char* mix = phase + Arena::round((size_t)r.p * (r.g.m + 1) * eb);
        double* a_host = ang + (size_t)b * 2 * QAOA_SERVE_MAX_P;
        double* a_dev = d_ang + (size_t)b * 2 * QAOA_SERVE_MAX_P;
        std::memcpy(a_host, r.gamma.data(), r.p * sizeof(double));
        std::memcpy(a_host + QAOA_SERVE_MAX_P, r.beta.data(), r.p * sizeof(double));
        std::memset(&cj[b], 0, sizeof(CoeffJob));
        cj[b].levels = r.p;
        cj[b].E1 = r.g.m + 1;
        cj[b].gamma = a_dev;
        cj[b].beta = a_dev + QAOA_SERVE_MAX_P;
        cj[b].phase = phase;
        cj[b].mix = mix;
        std::memset(&sj[b], 0, sizeof(SmallJob));
        sj[b].n = r.g.n;
        sj[b].levels = r.p;
        sj[b].E1 = r.g.m + 1;
        sj[b].synth = 1;
        sj[b].expect = 1;
        sj[b].store = 0;
        sj[b].init_amp = std::pow(2.0, -0.5 * r.g.n);
        for (int v = 0; v < kMaxN; ++v) sj[b].gmask[v] = v < r.g.n ? r.g.upper[v] : 0;
        sj[b].phase = phase;
        sj[b].mix = mix;
        sj[b].partials = d_res + b;
        nmax = std::max(nmax, r.g.n);
    }
    RunningBatch rb;
    rb.stream = pick_stream(sv, false);
    cudaStream_t stream = sv->streams[rb.stream];
    auto enqueue = [&]() -> qaoa_status {
        CUDA_TRY(cudaMemcpyAsync(head, stage, BL.upload, cudaMemcpyHostToDevice, stream));
        coeff_batch_kernel<real><<<B, 128, 0, stream>>>(reinterpret_cast<const CoeffJob*>(head + BL.coeff));
        CUDA_TRY(cudaGetLastError());
        small_batch_kernel<real><<<B, kSmallThreads, ((size_t)1 << nmax) * sizeof(C2), stream>>>(
            reinterpret_cast<const SmallJob*>(head + BL.small));
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(res_host, d_res, (size_t)B * sizeof(double2), cudaMemcpyDeviceToHost, stream));
        return QAOA_OK;
    };
    qaoa_status s = run_maybe_graph(sv, std::make_tuple(0, 0, 0, 0), stream, enqueue, &rb.exec);
    if (s == QAOA_OK) {
        rb.ev = take_event(sv);
        if (!rb.ev) s = fail(QAOA_ERR_CUDA, "cudaEventCreate failed");
        else if (cudaEventRecord(rb.ev, stream) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    }
    if (s != QAOA_OK) {
        release_graph(sv, rb.exec);
        return s;
    }
    sv->stream_load[rb.stream]++;
    rb.reqs = std::move(reqs);
    rb.offs = std::move(offs);
    rb.head_off = head_off;
    rb.head_bytes = BL.total;
    rb.staging = staging;
    rb.t_start = sv->now();
    bump(sv, &qaoa_server_stats::batches);
    bump(sv, &qaoa_server_stats::batched_requests, B);
    sv->batches.push_back(std::move(rb));
    return QAOA_OK;
}

// Whether a request runs in a packed mid-size launch: a complex64 forward request with unit
// weights whose state is tiled in two mixer groups (14 < n <= kMidMaxN) and p <= kMidMaxP.
bool serve_mid(const qaoa_server_s* sv, const SReq& r) {
    return sv->cfg.prec == QAOA_C64 && !r.grad && !r.g.weighted && !is_small(r.g.n, sv->cfg.prec) &&
           r.g.n <= kMidMaxN && r.p <= kMidMaxP;
}

// Packed launch of mid-size forward requests of one (n, p): every request keeps its own arena
// block (single_layout: state, phase tables, mixer entries), its pass arguments are the ones a
// lone run builds (fill_program_with, chunk_coeff_args) and its passes run the same compiled
// programs (pick_tile_batch_kernel), so each result equals the request run alone bit for bit.
// One upload of all descriptors, one coefficient launch, one launch per pass over the tiles of
// every request, one reduction launch, one download of the B results.  Returns
// QAOA_ERR_UNSUPPORTED (nothing enqueued) when a pass program has no packed kernel.
template <typename real>
qaoa_status dispatch_mid_batch(qaoa_server_s* sv, std::vector<SReq>& reqs, const std::vector<size_t>& offs,
                               const std::vector<size_t>& bytes, const std::vector<int>& slots, int staging) {
    constexpr int Q = PrecTraits<real>::Q, R = PrecTraits<real>::R;
    using C2 = typename C2T<real>::type;
    const int B = (int)reqs.size();
    const int n = reqs[0].g.n, p = reqs[0].p;
    const TileConfig tc = tile_config_for(sv->cfg.prec);
    const uint64_t tiles = 1ull << (n - Q);
    Plan plan;
    try {
        plan = plan_levels(n, tc, p, true, true);
    } catch (const std::exception& ex) {
        return fail(QAOA_ERR_UNSUPPORTED, ex.what());
    }
    const int passes = (int)plan.passes.size();
    if (passes > kMidMaxP + 1 || B > kMidMaxB) return fail(QAOA_ERR_UNSUPPORTED, "packed launch too large");
    const MidLayout ML = mid_layout(passes, B, tiles);
    unsigned char* stage = sv->pin_mid + (size_t)staging * mid_stage_bytes();
    TileArgs<Q>* targs = reinterpret_cast<TileArgs<Q>*>(stage + ML.targs);
    CoeffArgs* cargs = reinterpret_cast<CoeffArgs*>(stage + ML.cargs);
    double2* res_host = reinterpret_cast<double2*>(stage + ML.upload);
    RunningBatch rb;
    rb.stream = pick_stream(sv, false);
    cudaStream_t stream = sv->streams[rb.stream];
    unsigned gx = 1;
    for (int b = 0; b < B; ++b) {
        const SReq& r = reqs[b];
        const Layout L = single_layout(r.g, p, sv->cfg.prec, false, tiles);
        qaoa_state_s st;
        bind_request_state(sv, &st, r, sv->arena.base + offs[b], L, stream);
        for (int i = 0; i < passes; ++i) {
            TileArgs<Q>& a = targs[(size_t)i * B + b];
            std::memset(&a, 0, sizeof(a));
            fill_program_with(a, &st, plan.passes[i], st.groups, st.tc);
        }
        chunk_coeff_args(&st, p, r.gamma.data(), r.beta.data(), cargs[b]);
        gx = std::max(gx, coeff_grid(cargs[b]).x);
    }
    std::vector<TileBatchFn<real>> kfn(passes);
    for (int i = 0; i < passes; ++i) {
        kfn[i] = pick_tile_batch_kernel<real>(targs[(size_t)i * B]);
        if (!kfn[i]) return fail(QAOA_ERR_UNSUPPORTED, "no packed kernel for a pass program");
    }
    size_t head_off = 0;
    if (!sv->arena.alloc(ML.total, head_off)) return fail(QAOA_ERR_AGAIN, "no arena room for a packed launch");
    char* head = sv->arena.base + head_off;
    // the pass arguments name the head block's partials only now that it has an address
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < passes; ++i)
            targs[(size_t)i * B + b].partials = reinterpret_cast<double2*>(head + ML.partials) + (size_t)b * tiles;
    const TileArgs<Q>* d_targs = reinterpret_cast<const TileArgs<Q>*>(head + ML.targs);
    double2* d_partials = reinterpret_cast<double2*>(head + ML.partials);
    double2* d_results = reinterpret_cast<double2*>(head + ML.results);
    const size_t smem = (size_t)(1u << Q) * sizeof(C2);
    auto enqueue = [&]() -> qaoa_status {
        CUDA_TRY(cudaMemcpyAsync(head, stage, ML.upload, cudaMemcpyHostToDevice, stream));
        coeff_batch_args_kernel<real><<<dim3(gx, (unsigned)p, (unsigned)B), 256, 0, stream>>>(
            reinterpret_cast<const CoeffArgs*>(head + ML.cargs));
        CUDA_TRY(cudaGetLastError());
        for (int i = 0; i < passes; ++i) {
            kfn[i]<<<dim3((unsigned)tiles, (unsigned)B), 1u << (Q - R), smem, stream>>>(d_targs + (size_t)i * B);
            CUDA_TRY(cudaGetLastError());
        }
        finalize_batch_kernel<<<(unsigned)B, 1024, 0, stream>>>(d_partials, tiles, d_results);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(res_host, d_results, (size_t)B * sizeof(double2), cudaMemcpyDeviceToHost, stream));
        return QAOA_OK;
    };
    qaoa_status s = run_maybe_graph(sv, std::make_tuple(3, n, p, B), stream, enqueue, &rb.exec);
    if (s == QAOA_OK) {
        rb.ev = take_event(sv);
        if (!rb.ev) s = fail(QAOA_ERR_CUDA, "cudaEventCreate failed");
        else if (cudaEventRecord(rb.ev, stream) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    }
    if (s != QAOA_OK) {
        release_graph(sv, rb.exec);
        sv->arena.release(head_off, ML.total);
        return s;
    }
    sv->stream_load[rb.stream]++;
    rb.mid = true;
    rb.res_off = ML.upload;
    rb.reqs = std::move(reqs);
    rb.offs = offs;
    rb.bytes = bytes;
    rb.slots = slots;
    rb.head_off = head_off;
    rb.head_bytes = ML.total;
    rb.staging = staging;
    rb.t_start = sv->now();
    bump(sv, &qaoa_server_stats::batches);
    bump(sv, &qaoa_server_stats::batched_requests, B);
    bump(sv, &qaoa_server_stats::tiled_batches);
    bump(sv, &qaoa_server_stats::tiled_batched_requests, B);
    sv->batches.push_back(std::move(rb));
    return QAOA_OK;
}

void finish(qaoa_server_s* sv, const SReq& r, qaoa_result res) {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->done[r.ticket] = res;
    if (res.status == QAOA_OK) sv->stats.completed++;
    else sv->stats.failed++;
}

qaoa_result base_result(const SReq& r, double t_start, double t_done) {
    qaoa_result res;
    std::memset(&res, 0, sizeof(res));
    res.status = QAOA_OK;
    res.p = r.p;
    res.t_submit = r.t_submit;
    res.t_start = t_start;
    res.t_done = t_done;
    return res;
}

template <typename real>
bool scheduler_turn(qaoa_server_s* sv) {
    bool progress = false;
    // (1) retire completed work
    for (size_t i = 0; i < sv->running.size();) {
        Running& run = sv->running[i];
        const cudaError_t q = cudaEventQuery(run.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = sv->now();
        qaoa_result res = base_result(run.r, run.t_start, t);
        if (q != cudaSuccess) {
            res.status = QAOA_ERR_CUDA;
        } else {
            const double* host = sv->pin_single + (size_t)run.slot * (2 + 2 * QAOA_SERVE_MAX_P);
            res.expectation = host[0];
            res.norm = host[1];
            if (run.r.grad) {
                res.has_grad = 1;
                for (int k = 0; k < run.r.p; ++k) {
                    res.d_beta[k] = 2.0 * host[2 + k];
                    res.d_gamma[k] = 2.0 * host[2 + run.r.p + k];
                }
            }
        }
        finish(sv, run.r, res);
        release_graph(sv, run.exec);
        sv->event_pool.push_back(run.ev);
        sv->stream_load[run.stream]--;
        sv->free_single.push_back(run.slot);
        sv->arena.release(run.off, run.bytes);
        unbind_request_state(run.st);
        sv->inflight--;
        sv->running[i] = std::move(sv->running.back());
        sv->running.pop_back();
        progress = true;
    }
    for (size_t i = 0; i < sv->batches.size();) {
        RunningBatch& rb = sv->batches[i];
        const cudaError_t q = cudaEventQuery(rb.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = sv->now();
        const double2* res_host = reinterpret_cast<const double2*>(sv->pin_stage + (size_t)rb.staging * sv->stage_bytes +
                                                                   batch_layout(sv->cfg.max_batch).results);
        if (rb.mid)
            res_host = reinterpret_cast<const double2*>(sv->pin_mid + (size_t)rb.staging * mid_stage_bytes() + rb.res_off);
        for (size_t b = 0; b < rb.reqs.size(); ++b) {
            qaoa_result res = base_result(rb.reqs[b], rb.t_start, t);
            res.batched = 1;
            if (q != cudaSuccess) {
                res.status = QAOA_ERR_CUDA;
            } else {
                res.expectation = res_host[b].x;
                res.norm = res_host[b].y;
            }
            finish(sv, rb.reqs[b], res);
            sv->arena.release(rb.offs[b], rb.mid ? rb.bytes[b] : small_bytes(rb.reqs[b].g.m, rb.reqs[b].p, sv->cfg.prec));
            sv->inflight--;
        }
        for (int slot : rb.slots) sv->free_single.push_back(slot);
        release_graph(sv, rb.exec);
        sv->event_pool.push_back(rb.ev);
        sv->stream_load[rb.stream]--;
        (rb.mid ? sv->free_mid : sv->free_stage).push_back(rb.staging);
        sv->arena.release(rb.head_off, rb.head_bytes);
        sv->batches[i] = std::move(sv->batches.back());
        sv->batches.pop_back();
        progress = true;
    }
    // (2) requests still queued past their deadline complete with QAOA_ERR_TIMEOUT, unrun
    if (!sv->pending.empty()) {
        const double now = sv->now();
        for (auto it = sv->pending.begin(); it != sv->pending.end();) {
            if (it->deadline > 0.0 && now > it->deadline) {
                qaoa_result res = base_result(*it, now, now);
                res.status = QAOA_ERR_TIMEOUT;
                finish(sv, *it, res);
                bump(sv, &qaoa_server_stats::timed_out, 1);
                it = sv->pending.erase(it);
                progress = true;
            } else {
                ++it;
            }
        }
    }
    // (3) admission in arrival order, (4) packing, (5) dispatch
    std::vector<SReq> small;
    std::vector<size_t> small_offs;
    size_t head_off = 0;
    bool have_head = false;
    const size_t head_bytes = batch_layout(sv->cfg.max_batch).total;
    struct MidGroup {
        std::vector<SReq> reqs;
        std::vector<size_t> offs, bytes;
        std::vector<int> slots;
    };
    std::vector<MidGroup> mids;  // admitted mid-size requests, grouped by (n, p)
    const int mid_cap = std::min(sv->cfg.max_batch, kMidMaxB);
    while (!sv->pending.empty() && sv->inflight < sv->cfg.max_inflight) {
        SReq& r = sv->pending.front();
        if (serve_mid(sv, r)) {
            if (sv->free_single.empty()) break;
            const Layout L = single_layout(r.g, r.p, sv->cfg.prec, false, 1ull << (r.g.n - tile_config_for(sv->cfg.prec).Q));
            size_t off = 0;
            if (!sv->arena.alloc(L.total, off)) break;
            MidGroup* grp = nullptr;
            for (MidGroup& m : mids)
                if (m.reqs[0].g.n == r.g.n && m.reqs[0].p == r.p && (int)m.reqs.size() < mid_cap) grp = &m;
            if (!grp) {
                mids.emplace_back();
                grp = &mids.back();
            }
            grp->slots.push_back(sv->free_single.back());
            sv->free_single.pop_back();
            grp->offs.push_back(off);
            grp->bytes.push_back(L.total);
            grp->reqs.push_back(std::move(r));
            sv->pending.pop_front();
            sv->inflight++;
        } else if (serve_small(sv, r)) {
            if ((int)small.size() >= sv->cfg.max_batch) break;
            if (!have_head) {
                if (sv->free_stage.empty() || !sv->arena.alloc(head_bytes, head_off)) break;
                have_head = true;
            }
            size_t off = 0;
            if (!sv->arena.alloc(small_bytes(r.g.m, r.p, sv->cfg.prec), off)) break;
            small.push_back(std::move(r));
            small_offs.push_back(off);
            sv->pending.pop_front();
            sv->inflight++;
        } else {
            if (sv->free_single.empty()) break;
            const uint64_t ntiles = r.g.n > tile_config_for(sv->cfg.prec).Q
                                        ? (1ull << (r.g.n - tile_config_for(sv->cfg.prec).Q)) : 1ull;
            const Layout L = single_layout(r.g, r.p, sv->cfg.prec, r.grad, ntiles);
            size_t off = 0;
            if (!sv->arena.alloc(L.total, off)) break;
            const int slot = sv->free_single.back();
            sv->free_single.pop_back();
            SReq req = std::move(r);
            sv->pending.pop_front();
            sv->inflight++;
            const double t = sv->now();
            const qaoa_status s = dispatch_single<real>(sv, std::move(req), off, L, slot);
            if (s != QAOA_OK) {  // report the failure as the request's result (req was not consumed)
                qaoa_result res = base_result(req, t, t);
                res.status = s;
                sv->arena.release(off, L.total);
                sv->free_single.push_back(slot);
                sv->inflight--;
                finish(sv, req, res);
            }
        }
        progress = true;
    }
    if (!small.empty()) {
        const int staging = sv->free_stage.back();
        sv->free_stage.pop_back();
        std::vector<SReq> keep = small;  // for error reporting
        const qaoa_status s = dispatch_batch<real>(sv, std::move(small), std::move(small_offs), staging, head_off);
        if (s != QAOA_OK) {
            const double t = sv->now();
            for (size_t b = 0; b < keep.size(); ++b) {
                qaoa_result res = base_result(keep[b], t, t);
                res.status = s;
                finish(sv, keep[b], res);
                sv->arena.release(small_offs[b], small_bytes(keep[b].g.m, keep[b].p, sv->cfg.prec));
                sv->inflight--;
            }
            sv->arena.release(head_off, head_bytes);
            sv->free_stage.push_back(staging);
        }
        progress = true;
    } else if (have_head) {
        sv->arena.release(head_off, head_bytes);
    }
    // mid-size groups: packed when two or more share (n, p) and a staging slot and arena room for
    // the head are free, else each request runs alone in the block it was admitted with
    for (MidGroup& m : mids) {
        if (m.reqs.size() >= 2 && !sv->free_mid.empty()) {
            const int staging = sv->free_mid.back();
            sv->free_mid.pop_back();
            std::vector<SReq> keep = m.reqs;
            const qaoa_status s = dispatch_mid_batch<real>(sv, m.reqs, m.offs, m.bytes, m.slots, staging);
            if (s == QAOA_OK) continue;
            sv->free_mid.push_back(staging);
            m.reqs = std::move(keep);
            if (s != QAOA_ERR_AGAIN && s != QAOA_ERR_UNSUPPORTED) {  // a CUDA failure: report it
                const double t = sv->now();
                for (size_t b = 0; b < m.reqs.size(); ++b) {
                    qaoa_result res = base_result(m.reqs[b], t, t);
                    res.status = s;
                    finish(sv, m.reqs[b], res);
                    sv->arena.release(m.offs[b], m.bytes[b]);
                    sv->free_single.push_back(m.slots[b]);
                    sv->inflight--;
                }
                continue;
            }
        }
        for (size_t b = 0; b < m.reqs.size(); ++b) {
            const SReq& r0 = m.reqs[b];
            const Layout L = single_layout(r0.g, r0.p, sv->cfg.prec, false, 1ull << (r0.g.n - tile_config_for(sv->cfg.prec).Q));
            SReq req = std::move(m.reqs[b]);
            const double t = sv->now();
            const qaoa_status s = dispatch_single<real>(sv, std::move(req), m.offs[b], L, m.slots[b]);
            if (s != QAOA_OK) {
                qaoa_result res = base_result(req, t, t);
                res.status = s;
                sv->arena.release(m.offs[b], L.total);
                sv->free_single.push_back(m.slots[b]);
                sv->inflight--;
                finish(sv, req, res);
            }
        }
    }
    return progress;
}

template <typename real>
void scheduler_loop(qaoa_server_s* sv) {
    cudaSetDevice(sv->dev);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            while (!sv->queue.empty()) {
                sv->pending.push_back(std::move(sv->queue.front()));
                sv->queue.pop_front();
            }
            if (sv->stop) sv->pending.clear();  // not admitted yet: dropped
            if (sv->stop && sv->running.empty() && sv->batches.empty()) break;
        }
        const bool progress = scheduler_turn<real>(sv);
        if (!progress) {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->queue.empty() && !sv->stop)
                sv->cv.wait_for(lock, std::chrono::microseconds(sv->running.empty() && sv->batches.empty() ? 2000 : 20));
        }
    }
}

void server_free(qaoa_server_s* sv) {
    cudaSetDevice(sv->dev);
    for (cudaStream_t s : sv->streams)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    for (cudaEvent_t e : sv->event_pool) cudaEventDestroy(e);
    for (auto& kv : sv->graphs)
        for (auto& e : kv.second.execs) cudaGraphExecDestroy(e.first);
    if (sv->arena.base) cudaFree(sv->arena.base);
    if (sv->pin_single) cudaFreeHost(sv->pin_single);
    if (sv->pin_stage) cudaFreeHost(sv->pin_stage);
    if (sv->pin_mid) cudaFreeHost(sv->pin_mid);
    delete sv;
}

}  // namespace

extern "C" {

qaoa_status qaoa_server_create(const qaoa_server_config* cfg, qaoa_server* out) {
    if (!cfg || !out) return fail(QAOA_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->prec != QAOA_C64 && cfg->prec != QAOA_C128) return fail(QAOA_ERR_INVALID, "unknown precision");
    if (cfg->max_inflight < 1 || cfg->queue_capacity < 1 || cfg->max_batch < 1 || cfg->max_batch > 256 ||
        cfg->streams < 1 || cfg->streams > 64 || cfg->hbm_budget_bytes < ((size_t)1 << 20))
        return fail(QAOA_ERR_INVALID, "server configuration out of range");
    qaoa_server_s* sv = new (std::nothrow) qaoa_server_s;
    if (!sv) return fail(QAOA_ERR_OOM, "host allocation failed");
    sv->cfg = *cfg;
    sv->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&sv->dev);
    void* arena = nullptr;
    cudaError_t e = cudaMalloc(&arena, cfg->hbm_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return fail(QAOA_ERR_OOM, std::string("server arena allocation failed: ") + cudaGetErrorString(e));
    }
    sv->arena.init(static_cast<char*>(arena), cfg->hbm_budget_bytes);
    const int slots = cfg->max_inflight;
    sv->stage_bytes = batch_layout(cfg->max_batch).total;
    const int stages = std::max(2, std::min(16, cfg->streams * 2));
    e = cudaMallocHost(&sv->pin_single, (size_t)slots * (2 + 2 * QAOA_SERVE_MAX_P) * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&sv->pin_stage, (size_t)stages * sv->stage_bytes);
    if (e == cudaSuccess && cfg->prec == QAOA_C64) e = cudaMallocHost(&sv->pin_mid, (size_t)kMidStages * mid_stage_bytes());
    int prio_low = 0, prio_high = 0;  // stream 0 (the lane of GPU-filling requests) runs at the lowest
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    for (int i = 0; i < cfg->streams && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        const int prio = cfg->streams < 2 ? 0 : (i == 0 ? prio_low : prio_high);
        e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio);
        sv->streams.push_back(s);
        sv->stream_load.push_back(0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        server_free(sv);
        return fail(QAOA_ERR_OOM, std::string("server resources: ") + cudaGetErrorString(e));
    }
    for (int i = slots - 1; i >= 0; --i) sv->free_single.push_back(i);
    for (int i = stages - 1; i >= 0; --i) sv->free_stage.push_back(i);
    for (int i = kMidStages - 1; sv->pin_mid && i >= 0; --i) sv->free_mid.push_back(i);
    // kernel attributes are set here, outside any stream capture
    const qaoa_status st = cfg->prec == QAOA_C64 ? prepare_kernels<float>() : prepare_kernels<double>();
    if (st != QAOA_OK) {
        server_free(sv);
        return st;
    }
    sv->thr = cfg->prec == QAOA_C64 ? std::thread(scheduler_loop<float>, sv) : std::thread(scheduler_loop<double>, sv);
    *out = sv;
    return QAOA_OK;
}

qaoa_status qaoa_submit(qaoa_server sv, const qaoa_request* r, uint64_t* ticket) {
    if (!sv || !r || !ticket) return fail(QAOA_ERR_INVALID, "NULL argument");
    if (r->p < 1 || r->p > QAOA_SERVE_MAX_P) return fail(QAOA_ERR_INVALID, "p out of range for the server");
    if (!r->gamma || !r->beta) return fail(QAOA_ERR_INVALID, "angle array is NULL");
    if (!angles_ok(r->p, r->gamma) || !angles_ok(r->p, r->beta)) return fail(QAOA_ERR_INVALID, "non-finite angle");
    if (!(r->deadline_s >= 0.0) || !std::isfinite(r->deadline_s))
        return fail(QAOA_ERR_INVALID, "deadline must be finite and >= 0");
    SReq q;
    qaoa_status st = encode_graph(&r->graph, q.g);
    if (st != QAOA_OK) return st;
    q.p = r->p;
    q.gamma.assign(r->gamma, r->gamma + r->p);
    q.beta.assign(r->beta, r->beta + r->p);
    q.grad = r->want_grad != 0;
    const TileConfig tc = tile_config_for(sv->cfg.prec);
    const uint64_t ntiles = q.g.n > tc.Q ? (1ull << (q.g.n - tc.Q)) : 1ull;
    const size_t need = (!q.grad && !q.g.weighted && is_small(q.g.n, sv->cfg.prec)) ? small_bytes(q.g.m, q.p, sv->cfg.prec)
                                                                  : single_layout(q.g, q.p, sv->cfg.prec, q.grad, ntiles).total;
    if (need > sv->arena.size) return fail(QAOA_ERR_OOM, "request needs more device memory than the server's arena");
    std::lock_guard<std::mutex> lock(sv->mu);
    if ((int)sv->queue.size() >= sv->cfg.queue_capacity) {
        sv->stats.rejected_full++;
        return fail(QAOA_ERR_AGAIN, "server queue is full");
    }
    q.ticket = sv->next_ticket++;
    q.t_submit = sv->now();
    q.deadline = r->deadline_s > 0.0 ? q.t_submit + r->deadline_s : 0.0;
    *ticket = q.ticket;
    sv->live.insert(q.ticket);
    sv->queue.push_back(std::move(q));
    sv->stats.submitted++;
    sv->cv.notify_one();
    return QAOA_OK;
}

qaoa_status qaoa_poll(qaoa_server sv, uint64_t ticket, qaoa_result* out) {
    if (!sv || !out) return fail(QAOA_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->done.find(ticket);
    if (it != sv->done.end()) {
        *out = it->second;
        sv->done.erase(it);
        sv->live.erase(ticket);
        return QAOA_OK;
    }
    if (sv->live.count(ticket)) return QAOA_PENDING;
    return fail(QAOA_ERR_INVALID, "unknown ticket");
}

double qaoa_server_time(qaoa_server sv) { return sv ? sv->now() : 0.0; }

qaoa_status qaoa_server_stats_read(qaoa_server sv, qaoa_server_stats* out) {
    if (!sv || !out) return fail(QAOA_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
    return QAOA_OK;
}

qaoa_status qaoa_server_destroy(qaoa_server sv) {
    if (!sv) return QAOA_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->queue.clear();
        sv->cv.notify_all();
    }
    if (sv->thr.joinable()) sv->thr.join();
    server_free(sv);
    return QAOA_OK;
}

}  // extern "C"
