// Host runtime behind include/gsw.h: contexts, scratch management and the
// stage chain of one batch (plan -> fill -> 32-bit refill of overflowed pairs
// -> reversed fill -> banded traceback), all enqueued on the caller's stream.
#include "gsw_impl.cuh"

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace gsw;

namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace gsw {
int set_err(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int make_scoring(const int8_t *matrix, int32_t A, int32_t O, int32_t X, Scoring *sc) {
    if (!matrix) return set_err(GSW_EINVAL, "matrix is NULL");
    if (A < 1 || A > kMaxAlpha) return set_err(GSW_EINVAL, "alphabet %d not in [1, %d]", A, kMaxAlpha);
    if (X < 0 || O < X || O > 255) return set_err(GSW_EINVAL, "need 0 <= gap_extend <= gap_open <= 255 (got %d, %d)", O, X);
    std::memset(sc, 0, sizeof(*sc));
    sc->A = A;
    sc->O = O;
    sc->X = X;
    int wmax = -128, wmin = 127;
    for (int i = 0; i < A * A; i++) {
        if (matrix[i] < -127) return set_err(GSW_EINVAL, "matrix entry %d out of [-127, 127]", matrix[i]);
        sc->W[i] = matrix[i];
        wmax = std::max<int>(wmax, matrix[i]);
        wmin = std::min<int>(wmin, matrix[i]);
    }
    sc->wmax = wmax;
    sc->wmin = wmin;
    sc->dna4 = A == 4;
    sc->one = 1;
    std::memset(sc->fill_class, -1, sizeof(sc->fill_class));
    return GSW_OK;
}
}  // namespace gsw

namespace {

#define CUDA_TRY(x)                                                                            \
    do {                                                                                       \
        cudaError_t e__ = (x);                                                                 \
        if (e__ != cudaSuccess) return set_err(GSW_ECUDA, "%s: %s", #x, cudaGetErrorString(e__)); \
    } while (0)

#define GSW_TRY(x)              \
    do {                        \
        int r__ = (x);          \
        if (r__ != GSW_OK) return r__; \
    } while (0)

}  // namespace

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Host-side state of one pipeline run that the stages after the trace
// readback need (also saved with a captured graph).
struct PipeState {
    gsw::PlanBuffers pb;
    gsw::FillLaunch fl;
    size_t slots = 0, ncap = 0;
    int max_blocks = 0;
    long long *ring_prefix = nullptr;
    int *ring_final = nullptr, *ring_group = nullptr;
    long long ring_words = 0, ring_pool = 0;  // wide-band traceback sizes (stats)
    int ring_groups = 0;
    int launches = 0;
    int stage_done[GSW_NSTAGES] = {};
};

// One captured segment of the pipeline: replayed whenever the call repeats
// with the same key (pointers, sizes, flags, scoring, scratch), captured on
// the second call with that key.
struct GraphSeg {
    std::vector<uint8_t> key;
    bool seen = false;
    cudaGraphExec_t exec = nullptr;
    PipeState state;
    uint64_t used_at = 0;
};

// The segments of the keys seen last (least recently used ones make room),
// so calls whose shapes alternate (a server's length buckets) each replay
// their own graph.
constexpr size_t kGraphCacheEntries = 24;
struct GraphCache {
    std::vector<GraphSeg> e;
    uint64_t clock = 0;
};

struct gsw_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    int sms = 0;      // SMs the launches are sized for
    int sms_all = 0;  // SMs of the device
    cudaMemPool_t pool = nullptr;  // stream-ordered scratch allocations
    int8_t tune[GSW_TUNE_BUCKETS];  // fill class per query-row bucket (gsw_autotune), -1: default rule
    GraphCache seg[2];              // before and after the traceback readback
    bool graph_buckets = false;     // round shapes up to buckets so graphs repeat (serving)
    bool capturing = false;         // a segment is being captured: no allocation
    cudaStream_t st = nullptr;     // stream of the call in progress
    DevBuf plan_keys, plan_order, plan_small;
    DevBuf fill_cm, fill_bnd;
    DevBuf trace_dirs, trace_ops, band_scr, ring_meta;
    DevBuf misc;  // counters: trace head, cigar cursor, trace need, max lengths
    DevBuf io_q, io_t, io_qoff, io_toff, io_qlen, io_tlen, io_res, io_cigar, io_colmax, io_cmoff;
    DevBuf io_qp, io_tp;  // packed input staging (GSW_PACKED2 with GSW_HOST_IO)
    DevBuf prof_qoff, prof_qlen;
    void *host_small = nullptr;  // pinned readback area
    cudaEvent_t ev[GSW_NSTAGES + 1] = {};
    BandStreams aux = {};  // side streams of the band kernel's classes (created on first use)
    bool timing = false;
    int launches = 0;
    int stage_done[GSW_NSTAGES] = {};
    int graph_segments = 0;  // segments of the last call replayed from a graph
    long long cigar_words = 0;  // CIGAR words the last call needed
    long long internal = 0;     // records of the last call flagged kResInternal
    long long ring_words = 0, ring_pool = 0;  // wide-band traceback of the last call
    int ring_groups = 0;
};

struct gsw_profile {
    gsw_ctx *ctx;
    uint8_t *query;  // device
    int32_t qlen;
    Scoring sc;
};

namespace {

// Grows `b` to at least `need` bytes (never shrinks).  Allocation and release
// are stream-ordered on the call's stream (the context's own memory pool), so
// growing a buffer waits for no other stream's work: work queued on this
// stream that uses the old buffer runs before it is released.
int ensure(gsw_ctx *ctx, DevBuf &b, size_t need) {
    if (need <= b.bytes) return GSW_OK;
    if (ctx->capturing) return GSW_ESTATE;  // the segment runs without a graph
    need = std::max<size_t>(need, 256);
    if (b.p) {
        CUDA_TRY(cudaFreeAsync(b.p, ctx->st));
        ctx->used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (ctx->used + need > ctx->budget)
        return set_err(GSW_ENOMEM, "scratch of %zu bytes exceeds the context budget (%zu used of %zu)", need,
                       ctx->used, ctx->budget);
    cudaError_t e = cudaMallocFromPoolAsync(&b.p, need, ctx->pool, ctx->st);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return set_err(GSW_ENOMEM, "scratch allocation of %zu bytes: %s", need, cudaGetErrorString(e));
    }
    b.bytes = need;
    ctx->used += need;
    return GSW_OK;
}

void release(gsw_ctx *ctx, DevBuf &b) {
    if (ctx->capturing) return;  // ensure() then reports GSW_ESTATE
    if (b.p) cudaFreeAsync(b.p, ctx->st);
    ctx->used -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

// Bytes of budget left if buffers a and b were released.
size_t room(const gsw_ctx *ctx, const DevBuf &a, const DevBuf &b) {
    const size_t used = ctx->used - a.bytes - b.bytes;
    return ctx->budget > used ? ctx->budget - used : 0;
}

// Grows two buffers that are sized together, releasing both first when
// either must grow, so the budget never counts an old and a new copy.
int ensure2(gsw_ctx *ctx, DevBuf &a, size_t na, DevBuf &b, size_t nb) {
    if (na > a.bytes || nb > b.bytes) {
        if (ctx->capturing) return GSW_ESTATE;
        release(ctx, a);
        release(ctx, b);
    }
    int rc = ensure(ctx, a, na);
    return rc != GSW_OK ? rc : ensure(ctx, b, nb);
}


// device scratch layout of ctx->misc (64-bit words)
enum MiscSlot {
    kMiscTraceHead = 0,
    kMiscCursor = 1,
    kMiscInternal = 2,  // records flagged kResInternal (counted after the pipeline)
    kMiscValid = 3,
    kMiscNeed = 4,   // 2 words: anti-diagonal traceback (direction words, op words per pair)
    kMiscRing = 6,   // 3 words: wide-band traceback (total words, max words of a pair, max op words)
    kMiscStats = 12,   // 5 words: largest lengths, arena extents, bad lengths or offsets
    kMiscNeed16 = 17,  // 4 words: 16-bit rectangle traceback (direction words per group, per class)
    kMiscWords = 21
};

// Side streams and fork/join events of the band classes, created once per
// context outside any capture (the first call of a shape is never captured).
void destroy_aux(BandStreams &a) {
    for (int k = 0; k < 2; k++) {
        if (a.s[k]) cudaStreamDestroy(a.s[k]);
        if (a.join[k]) cudaEventDestroy(a.join[k]);
    }
    if (a.fork) cudaEventDestroy(a.fork);
    a = BandStreams{};
}

int ensure_aux(gsw_ctx *ctx) {
    if (ctx->aux.fork) return GSW_OK;
    if (ctx->capturing) return GSW_ESTATE;
    BandStreams a{};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaStreamCreateWithFlags(&a.s[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_aux(a);  // all or nothing: a later call tries again
        return set_err(GSW_ECUDA, "band side streams: %s", cudaGetErrorString(e));
    }
    ctx->aux = a;
    return GSW_OK;
}

// event e[k] marks the end of stage k-1 / start of stage k
int mark(gsw_ctx *ctx, int k, cudaStream_t st) {
    if (!ctx->timing) return GSW_OK;
    // while a segment is captured, an external record makes the graph record
    // the event each time it runs (a plain record would only order the capture)
    if (ctx->capturing) CUDA_TRY(cudaEventRecordWithFlags(ctx->ev[k], st, cudaEventRecordExternal));
    else CUDA_TRY(cudaEventRecord(ctx->ev[k], st));
    return GSW_OK;
}

template <class T>
void key_add(std::vector<uint8_t> &k, const T &v) {
    const uint8_t *p = reinterpret_cast<const uint8_t *>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

void key_buf(std::vector<uint8_t> &k, const DevBuf &b) {
    key_add(k, b.p);
    key_add(k, b.bytes);
}

// Runs body() on the stream, or replays it as a CUDA graph: a segment is
// captured on the second call with the same key (the first call sized every
// buffer, so the capture allocates nothing) and replayed while the key repeats.
// A segment that would have to grow a buffer while captured runs eagerly.
template <class F>
int run_segment(gsw_ctx *ctx, GraphCache &gc, const std::vector<uint8_t> &key, cudaStream_t st, PipeState &state,
                F body) {
    GraphSeg *g = nullptr;
    for (GraphSeg &x : gc.e)
        if (x.key == key) {
            g = &x;
            break;
        }
    if (g && g->exec) {
        CUDA_TRY(cudaGraphLaunch(g->exec, st));
        state = g->state;
        g->used_at = ++gc.clock;
        ctx->graph_segments++;
        return GSW_OK;
    }
    if (!g) {
        // first sighting: remember the key, run eagerly
        if (gc.e.size() >= kGraphCacheEntries) {
            size_t old = 0;
            for (size_t i = 1; i < gc.e.size(); i++)
                if (gc.e[i].used_at < gc.e[old].used_at) old = i;
            if (gc.e[old].exec) cudaGraphExecDestroy(gc.e[old].exec);
            gc.e.erase(gc.e.begin() + (long)old);
        }
        gc.e.emplace_back();
        g = &gc.e.back();
        g->key = key;
        g->seen = true;
        g->used_at = ++gc.clock;
        return body();
    }
    g->used_at = ++gc.clock;
    if (st == nullptr) return body();  // the legacy stream cannot be captured
    const PipeState before = state;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return body();
    }
    ctx->capturing = true;
    const int rc = body();
    ctx->capturing = false;
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &gr);
    cudaGraphExec_t ex = nullptr;
    if (rc == GSW_OK && e == cudaSuccess && gr && cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess) {
        cudaGraphDestroy(gr);
        g->exec = ex;
        g->state = state;
        CUDA_TRY(cudaGraphLaunch(ex, st));
        return GSW_OK;
    }
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();  // a failed capture leaves no error for the eager run
    state = before;
    return body();
}

// Shapes of a call rounded up to powers of four (at least 64) when the
// context replays graphs across calls of similar shape: the pipeline then
// sizes its scratch and launches from the bucket, which changes no result,
// and few buckets mean few captures.
uint64_t bucket_up(uint64_t x) {
    if (x == 0) return 0;
    uint64_t b = 64;
    while (b < x) b <<= 2;
    return b;
}

int run_pipeline(gsw_ctx *ctx, BatchView bv, const Scoring &sc, cudaStream_t st, int maxm, int maxn) {
    const int npairs = bv.npairs;
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(ctx->misc.p);
    unsigned long long *hs = reinterpret_cast<unsigned long long *>(ctx->host_small);
    PipeState S;
    std::vector<uint8_t> key;
    key.reserve(2048);
    key_add(key, bv);
    key_add(key, sc);
    key_add(key, maxm);
    key_add(key, maxn);
    key_add(key, st);
    key_add(key, ctx->sms);
    key_add(key, ctx->budget);
    key_add(key, ctx->used);
    key_add(key, ctx->timing);
    key_add(key, ctx->ev);
    for (const DevBuf *d : {&ctx->plan_keys, &ctx->plan_order, &ctx->plan_small, &ctx->fill_cm, &ctx->fill_bnd,
                            &ctx->band_scr, &ctx->ring_meta, &ctx->trace_dirs, &ctx->trace_ops, &ctx->misc})
        key_buf(key, *d);

    // ---- segment 1: fills, reverse, band kernel, traceback plan and needs
    auto seg1 = [&]() -> int {
        GSW_TRY(ensure(ctx, ctx->plan_keys, sizeof(int32_t) * (size_t)std::max(npairs, 1)));
        GSW_TRY(ensure(ctx, ctx->plan_order, sizeof(int32_t) * (size_t)std::max(npairs, 1)));
        const size_t small_words = 3 * (size_t)kPlanBins + 4 * kNumFillClasses + 8;
        GSW_TRY(ensure(ctx, ctx->plan_small, sizeof(int32_t) * small_words));
        int32_t *ps = reinterpret_cast<int32_t *>(ctx->plan_small.p);
        PlanBuffers &pb = S.pb;
        pb.keys = reinterpret_cast<int32_t *>(ctx->plan_keys.p);
        pb.order = reinterpret_cast<int32_t *>(ctx->plan_order.p);
        pb.hist = ps;
        pb.binoff = ps + kPlanBins;
        pb.cursor = ps + 2 * kPlanBins;
        pb.var_start = ps + 3 * kPlanBins;
        pb.task_lo = pb.var_start + kNumFillClasses + 1;
        pb.task_hi = pb.task_lo + kNumFillClasses;
        pb.ntasks = pb.task_hi + kNumFillClasses;
        pb.head = pb.ntasks + 1;

        // fill launch geometry and per-slot scratch
        const int warps_per_block = fill_block_threads() / 32;
        // columns per slot, a multiple of 4: every slot's max array starts on
        // a 16-byte boundary (the fill stores four 16-bit column maxima at a
        // time with one 8-byte store)
        S.ncap = ((size_t)std::max(maxn, 1) + 3) & ~(size_t)3;
        const size_t per_slot = S.ncap * sizeof(int32_t) + 2 * S.ncap * sizeof(int2);
        S.slots = (size_t)fill_slots(sc, ctx->sms);
        if (S.slots == 0) return set_err(GSW_ECUDA, "fill kernels cannot be resident");
        S.max_blocks = INT32_MAX;
        {
            // keep the scratch inside half of what the budget has left
            size_t have = room(ctx, ctx->fill_cm, ctx->fill_bnd);
            size_t cap_slots = have / 2 / per_slot;
            if (S.slots > cap_slots) {
                // a warp holds at most fill_max_pairs_per_warp() pairs
                const size_t per_warp = (size_t)fill_max_pairs_per_warp();
                S.max_blocks = (int)std::max<size_t>(1, cap_slots / (per_warp * warps_per_block));
                S.slots = (size_t)S.max_blocks * warps_per_block * per_warp;
            }
        }
        GSW_TRY(ensure2(ctx, ctx->fill_cm, S.slots * S.ncap * sizeof(int32_t), ctx->fill_bnd,
                        S.slots * 2 * S.ncap * sizeof(int2)));

        FillLaunch &fl = S.fl;
        fl.b = bv;
        fl.sc = sc;
        fl.bad_letters = reinterpret_cast<const int32_t *>(misc + kMiscValid);
        fl.plan.order = pb.order;
        fl.plan.var_start = pb.var_start;
        fl.plan.task_lo = pb.task_lo;
        fl.plan.task_hi = pb.task_hi;
        fl.plan.head = pb.head;
        fl.plan.ntasks = pb.ntasks;
        fl.scr.colmax = ctx->fill_cm.p;
        fl.scr.boundary = ctx->fill_bnd.p;
        fl.scr.ncap = (int32_t)S.ncap;
        fl.scr.nslots = (int32_t)S.slots;

        auto plan = [&](int32_t mode) -> int {
            cudaError_t e = launch_plan(bv, sc, mode, pb, st);
            if (e != cudaSuccess) return set_err(GSW_ECUDA, "plan: %s", cudaGetErrorString(e));
            S.launches += 3;
            return GSW_OK;
        };
        // a local score is at most min(m, n) x the largest matrix entry (gaps
        // never add), so when that stays within the 16-bit lanes' bound no
        // pair is flagged for the 32-bit refill
        const bool force_s32 = (bv.flags & GSW_FORCE_S32) != 0;
        const bool may_overflow = (long long)std::min(maxm, maxn) * std::max(sc.wmax, 0) > 32767 - sc.wmax;
        auto fill = [&](int32_t mode) -> int {
            fl.mode = mode;
            // the classes the plan can have used, from the longest query
            fl.class_mask = fill_class_mask(mode, maxm, sc, force_s32, force_s32 || may_overflow);
            cudaError_t e = launch_fill(fl, ctx->sms, S.max_blocks, st);
            if (e != cudaSuccess) return set_err(GSW_ECUDA, "fill: %s", cudaGetErrorString(e));
            S.launches += __builtin_popcount(fl.class_mask);
            return GSW_OK;
        };
        GSW_TRY(mark(ctx, 0, st));
        GSW_TRY(plan(kFillForward));
        GSW_TRY(mark(ctx, 1, st));
        GSW_TRY(fill(kFillForward));
        GSW_TRY(mark(ctx, 2, st));
        S.stage_done[0] = S.stage_done[1] = 1;
        // no pair flagged for the refill: its plan and launches are left out
        if (!force_s32 && may_overflow) {
            GSW_TRY(plan(kFillRerun));
            GSW_TRY(fill(kFillRerun));
            S.stage_done[2] = 1;
        }
        GSW_TRY(mark(ctx, 3, st));
        if (bv.flags & (GSW_BEGIN | GSW_CIGAR)) {
            // reversed fill in the ring kernels for pairs whose reverse band is wide
            GSW_TRY(plan(kFillReverse));
            GSW_TRY(fill(kFillReverse));
            S.stage_done[3] = 1;
        }
        GSW_TRY(mark(ctx, 4, st));
        if (bv.flags & (GSW_BEGIN | GSW_CIGAR)) {
            // thread-per-pair banded reverse and traceback for narrow bands
            // (the plan also hands a small batch's pairs to the warp tracebacks)
            GSW_TRY(plan(kPlanBand));
            if (!small_batch(bv)) {  // a small batch's band classes are empty
                const int rows_cap = std::min(std::max(maxm, 1), kBandMaxRows);
                // a quarter of what is left: the band scratch holds every row of
                // the pairs in flight
                const size_t have = room(ctx, ctx->band_scr, ctx->misc) + ctx->misc.bytes;  // budget left without band_scr
                const BandGrids bg = band_grids(rows_cap, ctx->sms, have / 4);
                if (bg.total_bytes > ctx->band_scr.bytes) release(ctx, ctx->band_scr);
                GSW_TRY(ensure(ctx, ctx->band_scr, bg.total_bytes));
                GSW_TRY(ensure_aux(ctx));
                CUDA_TRY(launch_band(bv, sc, pb, ctx->band_scr.p, bg, st, ctx->aux));
                S.launches += 3;
            }
            S.stage_done[4] = 1;
        }
        GSW_TRY(mark(ctx, 5, st));
        if (bv.flags & GSW_CIGAR) {
            // tracebacks for the pairs the band kernel left (band wider than 32
            // or more than 4096 rows): anti-diagonal warp kernel up to 512
            // diagonals, CTA strip kernel beyond; their scratch is sized from
            // the needs read back after this segment
            GSW_TRY(plan(kPlanTrace));
            CUDA_TRY(launch_trace_need(bv, sc, misc + kMiscNeed, misc + kMiscNeed16, st));
            const size_t meta_bytes = sizeof(long long) * ((size_t)npairs + 1) + sizeof(int) * ((size_t)npairs + 4);
            GSW_TRY(ensure(ctx, ctx->ring_meta, meta_bytes));
            S.ring_prefix = reinterpret_cast<long long *>(ctx->ring_meta.p);
            S.ring_final = reinterpret_cast<int *>(S.ring_prefix + npairs + 1);
            S.ring_group = S.ring_final + npairs;
            CUDA_TRY(launch_ring_needs(bv, sc, pb.order, pb.var_start, S.ring_prefix, misc + kMiscRing, st));
            CUDA_TRY(cudaMemsetAsync(S.ring_group, 0, 3 * sizeof(int), st));
            S.launches += 2;
            CUDA_TRY(cudaMemcpyAsync(hs, misc + kMiscNeed, (kMiscWords - kMiscNeed) * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st));
        }
        return GSW_OK;
    };
    GSW_TRY(run_segment(ctx, ctx->seg[0], key, st, S, seg1));

    if (bv.flags & GSW_CIGAR) {
        CUDA_TRY(cudaStreamSynchronize(st));
        // [0, 1] anti-diagonal, [2, 4] ring, [13, 16] 16-bit rectangle classes (others unused here)
        unsigned long long need[kMiscWords - kMiscNeed];
        std::memcpy(need, hs, sizeof(need));
        for (int k = 5; k < kMiscNeed16 - kMiscNeed; k++) need[k] = 0;
        if (ctx->graph_buckets)
            for (unsigned long long &x : need) x = bucket_up(x);
        std::vector<uint8_t> key2 = key;
        key_add(key2, need);
        for (const DevBuf *d : {&ctx->fill_bnd, &ctx->trace_dirs, &ctx->trace_ops, &ctx->ring_meta})
            key_buf(key2, *d);
        key_add(key2, ctx->used);

        // ---- segment 2: the tracebacks, sized from the needs
        auto seg2 = [&]() -> int {
            const PlanBuffers &pb = S.pb;
            // anti-diagonal kernel (<= 512 diagonals): direction and op words per warp
            const long long ad_dir = (long long)need[0], ad_ops = std::max<long long>((long long)need[1], 64);
            int ad_grid = 0;
            size_t max_dir = 0, max_ops = 0;
            const int wpb = trace_block_threads() / 32;
            if (ad_dir > 0) {
                const size_t have = room(ctx, ctx->trace_dirs, ctx->trace_ops) / 2;
                const size_t per_warp = (size_t)(ad_dir + ad_ops) * sizeof(uint32_t);
                int warps = (int)std::min<size_t>((size_t)ctx->sms * 16 * wpb, std::max<size_t>(1, have / per_warp));
                warps = std::max(wpb, warps - warps % wpb);
                ad_grid = warps / wpb;
                max_dir = (size_t)warps * (size_t)ad_dir;
                max_ops = (size_t)warps * (size_t)ad_ops;
            }
            // 16-bit rectangle kernel: per class, 4 groups per warp, direction
            // and op words per group (the classes run one after the other)
            T16Scratch t16{};
            bool any16 = false;
            {
                const size_t have = room(ctx, ctx->trace_dirs, ctx->trace_ops) / 2;
                for (int v = 0; v < kTraceT16Classes; v++) {
                    // 16-byte aligned group areas
                    const long long dw = ((long long)need[kMiscNeed16 - kMiscNeed + v] + 3) & ~3LL;
                    if (dw <= 0) continue;
                    const size_t per_warp = 4 * (size_t)(dw + ad_ops) * sizeof(uint32_t);
                    const int w = (int)std::min<size_t>((size_t)t16_max_warps(sc, ctx->sms, v),
                                                        std::max<size_t>(1, have / per_warp));
                    if (w <= 0) continue;
                    t16.dir_words[v] = dw;
                    t16.warps[v] = w;
                    max_dir = std::max(max_dir, (size_t)w * 4 * (size_t)dw);
                    max_ops = std::max(max_ops, (size_t)w * 4 * (size_t)ad_ops);
                    any16 = true;
                }
            }
            // wide bands: the pool of direction words, groups of pairs that fit it
            const unsigned long long ring_total = need[2], ring_max = need[3], ring_ops = need[4];
            size_t ring_pool = 0, ring_walk_warps = 0;
            if (ring_total > 0) {
                ring_walk_warps = (size_t)ctx->sms * 16;
                const size_t have_all = room(ctx, ctx->trace_dirs, ctx->trace_ops);
                const size_t ops_bytes = ring_walk_warps * (size_t)ring_ops * sizeof(uint32_t);
                size_t cap = have_all > ops_bytes ? (have_all - ops_bytes) / 2 / sizeof(uint32_t) : 0;
                ring_pool = (size_t)std::min<unsigned long long>(ring_total, cap);
                if (ring_pool < ring_max)
                    return set_err(GSW_ENOMEM, "wide-band traceback of one pair needs %llu words", ring_max);
                max_dir = std::max(max_dir, ring_pool);
                max_ops = std::max(max_ops, ring_walk_warps * (size_t)ring_ops);
            }
            if (max_dir > 0) {
                GSW_TRY(ensure2(ctx, ctx->trace_dirs, max_dir * sizeof(uint32_t), ctx->trace_ops,
                                max_ops * sizeof(uint32_t)));
                if (any16) {
                    t16.dirs = reinterpret_cast<uint32_t *>(ctx->trace_dirs.p);
                    t16.ops = reinterpret_cast<uint32_t *>(ctx->trace_ops.p);
                    t16.op_words = ad_ops;
                    t16.order = pb.order;
                    t16.var_start = pb.var_start;
                    t16.head = pb.head;
                    CUDA_TRY(launch_trace16(bv, sc, t16, ctx->sms, st));
                    for (int v = 0; v < kTraceT16Classes; v++) S.launches += t16.warps[v] > 0 ? 1 : 0;
                }
                if (ad_grid > 0) {
                    TraceScratch ts;
                    ts.dirs = reinterpret_cast<uint32_t *>(ctx->trace_dirs.p);
                    ts.dir_words = ad_dir;
                    ts.ops = reinterpret_cast<uint32_t *>(ctx->trace_ops.p);
                    ts.op_words = ad_ops;
                    ts.order = pb.order;
                    ts.var_start = pb.var_start;
                    CUDA_TRY(launch_trace_ad(bv, sc, ts, ad_grid, st));
                    S.launches += 4;
                }
                if (ring_total > 0) {
                    RingLaunchArgs ra;
                    ra.b = bv;
                    ra.sc = sc;
                    ra.order = pb.order;
                    ra.var_start = pb.var_start;
                    ra.prefix = S.ring_prefix;
                    ra.final_h = S.ring_final;
                    ra.group = S.ring_group;
                    ra.pool = reinterpret_cast<uint32_t *>(ctx->trace_dirs.p);
                    ra.pool_words = (long long)ring_pool;
                    ra.bnd = reinterpret_cast<int2 *>(ctx->fill_bnd.p);
                    ra.bnd_stride = 2 * (long long)S.ncap;
                    ra.slots = (int)S.slots;
                    ra.ops = reinterpret_cast<uint32_t *>(ctx->trace_ops.p);
                    ra.op_words = (long long)ring_ops;
                    ra.walk_warps = (int)ring_walk_warps;
                    // every group but the last fills more than pool - max_pair
                    const unsigned long long per = ring_pool > ring_max ? ring_pool - ring_max : 1;
                    const unsigned long long groups =
                        ring_total <= ring_pool ? 1 : (ring_total + per - 1) / per + 1;
                    for (unsigned long long gi = 0; gi < groups; gi++) {
                        CUDA_TRY(launch_ring_group(ra, ctx->sms, st));
                        S.launches += 4;
                    }
                    S.ring_words = (long long)ring_total;
                    S.ring_pool = (long long)ring_pool;
                    S.ring_groups = (int)groups;
                }
            }
            S.stage_done[5] = 1;
            GSW_TRY(mark(ctx, 6, st));
            return GSW_OK;
        };
        GSW_TRY(run_segment(ctx, ctx->seg[1], key2, st, S, seg2));
    } else {
        GSW_TRY(mark(ctx, 6, st));
    }
    ctx->launches += S.launches;
    ctx->ring_words = S.ring_words;
    ctx->ring_pool = S.ring_pool;
    ctx->ring_groups = S.ring_groups;
    for (int k = 0; k < GSW_NSTAGES; k++) ctx->stage_done[k] |= S.stage_done[k];
    return GSW_OK;
}

int check_common(gsw_ctx *ctx, int32_t npairs, uint32_t flags) {
    if (!ctx) return set_err(GSW_EINVAL, "context is NULL");
    if (npairs < 0) return set_err(GSW_EINVAL, "npairs < 0");
    if (flags & ~(GSW_BEGIN | GSW_CIGAR | GSW_COLMAX | GSW_HOST_IO | GSW_FORCE_S32 | GSW_PLAIN | GSW_TIMING |
                  GSW_PACKED2))
        return set_err(GSW_EINVAL, "unknown flag bits 0x%x", flags);
    if ((flags & GSW_PACKED2) && (flags & GSW_PLAIN)) return set_err(GSW_EINVAL, "GSW_PACKED2 with GSW_PLAIN");
    return GSW_OK;
}

int batch_impl(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
               const uint8_t *t, const int64_t *t_off, const int32_t *t_len, const Scoring &sc_in, uint32_t flags,
               int32_t mask_len, gsw_result *results, uint32_t *cigar, int64_t cigar_capacity, int32_t *colmax,
               const int64_t *colmax_off, cudaStream_t st) {
    GSW_TRY(check_common(ctx, npairs, flags));
    Scoring sc = sc_in;
    std::memcpy(sc.fill_class, ctx->tune, sizeof(sc.fill_class));
    if (flags & GSW_CIGAR) flags |= GSW_BEGIN;
    if (npairs == 0) return GSW_OK;
    if (!q || !q_off || !q_len || !t || !t_off || !t_len || !results)
        return set_err(GSW_EINVAL, "NULL input or result pointer");
    if ((flags & GSW_CIGAR) && (!cigar && cigar_capacity > 0)) return set_err(GSW_EINVAL, "cigar is NULL");
    if (cigar_capacity < 0) return set_err(GSW_EINVAL, "cigar_capacity < 0");
    if ((flags & GSW_COLMAX) && (!colmax || !colmax_off)) return set_err(GSW_EINVAL, "colmax output missing");
    if (mask_len > (1 << 30)) return set_err(GSW_EINVAL, "mask_len too large");
    CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->st = st;
    GSW_TRY(ensure(ctx, ctx->misc, kMiscWords * sizeof(unsigned long long)));
    ctx->launches = 0;
    ctx->graph_segments = 0;
    ctx->cigar_words = 0;
    ctx->internal = 0;
    ctx->ring_words = ctx->ring_pool = 0;
    ctx->ring_groups = 0;
    for (int k = 0; k < GSW_NSTAGES; k++) ctx->stage_done[k] = 0;
    ctx->timing = (flags & GSW_TIMING) != 0;
    if (ctx->timing && !ctx->ev[0])
        for (int k = 0; k <= GSW_NSTAGES; k++) CUDA_TRY(cudaEventCreate(&ctx->ev[k]));
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(ctx->misc.p);
    BatchView bv;
    std::memset(&bv, 0, sizeof(bv));
    bv.npairs = npairs;
    bv.flags = flags;
    bv.mask_len = mask_len;
    bv.cigar_cap = cigar_capacity;
    bv.cigar_cursor = misc + kMiscCursor;
    int maxm = 0, maxn = 0;
    int64_t cmext = 0;  // host I/O: colmax words from 0 to the end of the last pair's range
    const bool hio = (flags & GSW_HOST_IO) != 0;
    unsigned long long *hstat = reinterpret_cast<unsigned long long *>(ctx->host_small);
    // the batch's sizes and the checks of its lengths and offsets, on the
    // device in one pass (one 40-byte readback before anything is sized)
    auto batch_stats = [&](const int64_t *qo, const int32_t *ql, const int64_t *to, const int32_t *tl) -> int {
        CUDA_TRY(launch_batch_stats(qo, ql, to, tl, npairs, misc + kMiscStats, st));
        ctx->launches += 1;
        CUDA_TRY(cudaMemcpyAsync(hstat, misc + kMiscStats, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return GSW_OK;
    };
    if (hio) {
        // offsets and lengths first; the arenas once their extents are known
        GSW_TRY(ensure(ctx, ctx->io_qoff, sizeof(int64_t) * npairs));
        GSW_TRY(ensure(ctx, ctx->io_toff, sizeof(int64_t) * npairs));
        GSW_TRY(ensure(ctx, ctx->io_qlen, sizeof(int32_t) * npairs));
        GSW_TRY(ensure(ctx, ctx->io_tlen, sizeof(int32_t) * npairs));
        CUDA_TRY(cudaMemcpyAsync(ctx->io_qoff.p, q_off, sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(ctx->io_toff.p, t_off, sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(ctx->io_qlen.p, q_len, sizeof(int32_t) * npairs, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(ctx->io_tlen.p, t_len, sizeof(int32_t) * npairs, cudaMemcpyHostToDevice, st));
        GSW_TRY(batch_stats((const int64_t *)ctx->io_qoff.p, (const int32_t *)ctx->io_qlen.p,
                            (const int64_t *)ctx->io_toff.p, (const int32_t *)ctx->io_tlen.p));
        if (hstat[4]) {
            for (int32_t p = 0; p < npairs; p++) {
                if (q_len[p] < 0 || t_len[p] < 0 || q_len[p] >= (1 << 24) || t_len[p] >= (1 << 24))
                    return set_err(GSW_EINVAL, "pair %d: length out of [0, 2^24)", p);
                if (q_off[p] < 0 || t_off[p] < 0) return set_err(GSW_EINVAL, "pair %d: negative offset", p);
            }
        }
        maxm = (int)hstat[0];
        maxn = (int)hstat[1];
        const int64_t qext = (int64_t)hstat[2], text = (int64_t)hstat[3];
        if (flags & GSW_COLMAX)
            for (int32_t p = 0; p < npairs; p++) {
                if (colmax_off[p] < 0) return set_err(GSW_EINVAL, "pair %d: negative colmax offset", p);
                cmext = std::max<int64_t>(cmext, colmax_off[p] + t_len[p]);
            }
        GSW_TRY(ensure(ctx, ctx->io_q, (size_t)std::max<int64_t>(qext, 1)));
        GSW_TRY(ensure(ctx, ctx->io_t, (size_t)std::max<int64_t>(text, 1)));
        GSW_TRY(ensure(ctx, ctx->io_res, sizeof(gsw_result) * npairs));
        if (flags & GSW_CIGAR) GSW_TRY(ensure(ctx, ctx->io_cigar, sizeof(uint32_t) * (size_t)std::max<int64_t>(cigar_capacity, 1)));
        if (flags & GSW_COLMAX) {
            GSW_TRY(ensure(ctx, ctx->io_colmax, sizeof(int32_t) * (size_t)std::max<int64_t>(cmext, 1)));
            GSW_TRY(ensure(ctx, ctx->io_cmoff, sizeof(int64_t) * npairs));
        }
        if (flags & GSW_PACKED2) {
            // packed bytes in, one byte per letter on the device
            const size_t qb = (size_t)(qext + 3) / 4, tb = (size_t)(text + 3) / 4;
            GSW_TRY(ensure(ctx, ctx->io_qp, std::max<size_t>(qb, 1)));
            GSW_TRY(ensure(ctx, ctx->io_tp, std::max<size_t>(tb, 1)));
            CUDA_TRY(cudaMemcpyAsync(ctx->io_qp.p, q, qb, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(ctx->io_tp.p, t, tb, cudaMemcpyHostToDevice, st));
            CUDA_TRY(launch_unpack2((const uint8_t *)ctx->io_qp.p, (uint8_t *)ctx->io_q.p, qext, st));
            CUDA_TRY(launch_unpack2((const uint8_t *)ctx->io_tp.p, (uint8_t *)ctx->io_t.p, text, st));
            ctx->launches += 2;
        } else {
            CUDA_TRY(cudaMemcpyAsync(ctx->io_q.p, q, qext, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(ctx->io_t.p, t, text, cudaMemcpyHostToDevice, st));
        }
        if (flags & GSW_COLMAX) {
            CUDA_TRY(cudaMemcpyAsync(ctx->io_cmoff.p, colmax_off, sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, st));
            // the staging copy starts as the caller's buffer, so the words
            // between the pairs' ranges come back unchanged
            CUDA_TRY(cudaMemcpyAsync(ctx->io_colmax.p, colmax, sizeof(int32_t) * cmext, cudaMemcpyHostToDevice, st));
        }
        bv.q = (const uint8_t *)ctx->io_q.p;
        bv.t = (const uint8_t *)ctx->io_t.p;
        bv.q_off = (const int64_t *)ctx->io_qoff.p;
        bv.t_off = (const int64_t *)ctx->io_toff.p;
        bv.q_len = (const int32_t *)ctx->io_qlen.p;
        bv.t_len = (const int32_t *)ctx->io_tlen.p;
        bv.res = (gsw_result *)ctx->io_res.p;
        bv.cigar = (uint32_t *)ctx->io_cigar.p;
        bv.colmax = (int32_t *)ctx->io_colmax.p;
        bv.colmax_off = (const int64_t *)ctx->io_cmoff.p;
    } else {
        bv.q = q;
        bv.t = t;
        bv.q_off = q_off;
        bv.t_off = t_off;
        bv.q_len = q_len;
        bv.t_len = t_len;
        bv.res = results;
        bv.cigar = cigar;
        bv.colmax = colmax;
        bv.colmax_off = colmax_off;
        GSW_TRY(batch_stats(q_off, q_len, t_off, t_len));
        if (hstat[4]) return set_err(GSW_EINVAL, "a length is outside [0, 2^24) or an offset is negative");
        maxm = (int)hstat[0];
        maxn = (int)hstat[1];
        if (flags & GSW_PACKED2) {
            // expand the caller's packed arenas into context scratch
            const unsigned long long ext[2] = {hstat[2], hstat[3]};
            GSW_TRY(ensure(ctx, ctx->io_q, (size_t)std::max<unsigned long long>(ext[0], 1)));
            GSW_TRY(ensure(ctx, ctx->io_t, (size_t)std::max<unsigned long long>(ext[1], 1)));
            CUDA_TRY(launch_unpack2(q, (uint8_t *)ctx->io_q.p, (long long)ext[0], st));
            CUDA_TRY(launch_unpack2(t, (uint8_t *)ctx->io_t.p, (long long)ext[1], st));
            ctx->launches += 2;
            bv.q = (const uint8_t *)ctx->io_q.p;
            bv.t = (const uint8_t *)ctx->io_t.p;
        }
    }
    if (ctx->graph_buckets) {
        maxm = (int)bucket_up((uint64_t)maxm);
        maxn = (int)bucket_up((uint64_t)maxn);
    }
    CUDA_TRY(cudaMemsetAsync(misc + kMiscCursor, 0, 2 * sizeof(unsigned long long), st));  // cursor, internal
    if ((flags & GSW_PACKED2) && sc.A >= 4) {
        // 2-bit letters are 0..3: valid under any matrix of 4 or more letters
        CUDA_TRY(cudaMemsetAsync(misc + kMiscValid, 0, sizeof(int32_t), st));
    } else {
        CUDA_TRY(launch_validate(bv, sc, reinterpret_cast<int32_t *>(misc + kMiscValid), st));
        ctx->launches += 1;
    }
    GSW_TRY(run_pipeline(ctx, bv, sc, st, maxm, maxn));

    // completion: invalid letters, internal checks, CIGAR space
    CUDA_TRY(launch_count_flag(bv.res, npairs, kResInternal, misc + kMiscInternal, st));
    ctx->launches += 1;
    unsigned long long *hs = reinterpret_cast<unsigned long long *>(ctx->host_small);
    CUDA_TRY(cudaMemcpyAsync(hs, misc + kMiscCursor, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hs + 2, misc + kMiscValid, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if (hio) {
        CUDA_TRY(cudaMemcpyAsync(results, bv.res, sizeof(gsw_result) * npairs, cudaMemcpyDeviceToHost, st));
        if (flags & GSW_COLMAX)
            CUDA_TRY(cudaMemcpyAsync(colmax, bv.colmax, sizeof(int32_t) * cmext, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned long long used_words = hs[0];
    const unsigned long long internal = hs[1];
    const int bad_letters = (int)(hs[2] & 0xFFFFFFFFu);
    ctx->cigar_words = (flags & GSW_CIGAR) ? (long long)used_words : 0;
    if (hio && (flags & GSW_CIGAR) && cigar_capacity > 0) {
        const size_t n = (size_t)std::min<unsigned long long>(used_words, (unsigned long long)cigar_capacity);
        if (n) {
            CUDA_TRY(cudaMemcpyAsync(cigar, bv.cigar, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
    ctx->internal = (long long)internal;
    switch (batch_status(bad_letters, internal, (flags & GSW_CIGAR) != 0, used_words, cigar_capacity)) {
    case GSW_EINVAL: return set_err(GSW_EINVAL, "a letter code is >= the alphabet size (%d)", sc.A);
    case GSW_EINTERNAL:
        return set_err(GSW_EINTERNAL, "%llu pairs failed a consistency check of the kernels (GSW_RES_INTERNAL)",
                       internal);
    case GSW_ECIGAR_SPACE:
        return set_err(GSW_ECIGAR_SPACE, "CIGAR words needed %llu > capacity %lld", used_words,
                       (long long)cigar_capacity);
    default: return GSW_OK;
    }
}

// Baseline without batching: every pair goes through its own launch
// sequence (plan, fill, refill, reverse, traceback) and is waited for before
// the next one starts, as a caller aligning one pair per call would.
int plain_impl(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
               const uint8_t *t, const int64_t *t_off, const int32_t *t_len, const Scoring &sc, uint32_t flags,
               int32_t mask_len, gsw_result *results, uint32_t *cigar, int64_t cigar_capacity, int32_t *colmax,
               const int64_t *colmax_off, cudaStream_t st) {
    GSW_TRY(check_common(ctx, npairs, flags));
    flags &= ~GSW_PLAIN;
    if ((flags & GSW_CIGAR) && (flags & GSW_HOST_IO) == 0)
        return set_err(GSW_EINVAL, "GSW_PLAIN with GSW_CIGAR needs GSW_HOST_IO (per-pair CIGAR offsets)");
    int64_t cig_used = 0;
    int rc_internal = GSW_OK;
    for (int32_t p = 0; p < npairs; p++) {
        uint32_t *cg = cigar ? cigar + cig_used : nullptr;
        const int64_t cap = cigar ? cigar_capacity - cig_used : 0;
        int rc = batch_impl(ctx, 1, q, q_off + p, q_len + p, t, t_off + p, t_len + p, sc, flags, mask_len,
                            results + p, cg, cap, colmax, colmax_off ? colmax_off + p : nullptr, st);
        if (rc == GSW_EINTERNAL) {  // the record is complete apart from its flagged parts
            rc_internal = rc;
            rc = GSW_OK;
        }
        if (rc != GSW_OK) return rc;
        if ((flags & GSW_CIGAR) && results[p].cigar_len > 0) {
            results[p].cigar_off += cig_used;
            cig_used += results[p].cigar_len;
        }
    }
    return rc_internal != GSW_OK ? set_err(rc_internal, "pairs failed a consistency check (GSW_RES_INTERNAL)")
                                 : GSW_OK;
}

}  // namespace

extern "C" {

const char *gsw_version(void) { return "gsw 0.1 (sm_103a)"; }

const char *gsw_strerror(int code) {
    switch (code) {
    case GSW_OK: return "ok";
    case GSW_EINVAL: return "invalid argument";
    case GSW_ENOMEM: return "out of memory or over budget";
    case GSW_ECUDA: return "CUDA error";
    case GSW_ETIMEDOUT: return "timed out";
    case GSW_ECIGAR_SPACE: return "CIGAR buffer too small";
    case GSW_EOVERFLOW: return "score overflow";
    case GSW_ENOTFOUND: return "not found";
    case GSW_ESTATE: return "invalid state";
    case GSW_EINTERNAL: return "internal consistency check failed";
    default: return "unknown error";
    }
}

const char *gsw_last_error(void) { return g_err; }

int gsw_last_stats(const gsw_ctx *ctx, gsw_stats *out) {
    if (!ctx || !out) return set_err(GSW_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->kernel_launches = ctx->launches;
    out->graph_segments = ctx->graph_segments;
    out->cigar_words = ctx->cigar_words;
    out->ring_words = ctx->ring_words;
    out->ring_pool_words = ctx->ring_pool;
    out->ring_groups = ctx->ring_groups;
    out->internal_pairs = (int32_t)ctx->internal;
    if (!ctx->timing || !ctx->ev[0]) return GSW_OK;
    out->timed = 1;
    // stage k spans events k..k+1, except: [0] = e0..e1, [1] = e1..e2, [2] = e2..e3,
    // [3] = e3..e4, [4] = e4..e5, [5] = e5..e6, [6] = e0..e6
    // a failed query must not leave its error for the next call's launch checks
    auto elapsed = [](cudaEvent_t a, cudaEvent_t b) -> float {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            return 0.f;
        }
        return ms;
    };
    for (int k = 0; k < 6; k++)
        if (ctx->stage_done[k]) out->stage_ms[k] = elapsed(ctx->ev[k], ctx->ev[k + 1]);
    out->stage_ms[6] = elapsed(ctx->ev[0], ctx->ev[6]);
    return GSW_OK;
}

int gsw_context_create(int device, size_t mem_budget_bytes, gsw_ctx **out) {
    if (!out) return set_err(GSW_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_err(GSW_EINVAL, "device %d of %d", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    gsw_ctx *c = new (std::nothrow) gsw_ctx();
    if (!c) return set_err(GSW_ENOMEM, "host allocation");
    c->device = device;
    c->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)4 << 30);
    std::memset(c->tune, -1, sizeof(c->tune));
    cudaError_t e = cudaDeviceGetAttribute(&c->sms_all, cudaDevAttrMultiProcessorCount, device);
    c->sms = c->sms_all;
    if (e == cudaSuccess) {
        // the context's own pool keeps its memory between calls (no release
        // at synchronisation), so scratch stays resident
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&c->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_small, 4096);
    if (e != cudaSuccess) {
        delete c;
        return set_err(GSW_ECUDA, "context setup: %s", cudaGetErrorString(e));
    }
    *out = c;
    return GSW_OK;
}

}  // extern "C"

namespace gsw {
int context_device(const gsw_ctx *ctx) { return ctx->device; }
void context_set_graph_buckets(gsw_ctx *ctx, bool on) { ctx->graph_buckets = on; }
}  // namespace gsw

extern "C" {

int gsw_context_set_tune(gsw_ctx *c, const gsw_tune *t) {
    if (!c) return set_err(GSW_EINVAL, "context is NULL");
    if (!t) {
        std::memset(c->tune, -1, sizeof(c->tune));
        return GSW_OK;
    }
    for (int b = 0; b < GSW_TUNE_BUCKETS; b++)
        if (t->fill_class[b] < -1 || t->fill_class[b] > 13 || t->fill_class[b] == 7)
            return set_err(GSW_EINVAL, "fill class %d of bucket %d", t->fill_class[b], b);
    std::memcpy(c->tune, t->fill_class, sizeof(c->tune));
    return GSW_OK;
}

int gsw_context_set_sm_limit(gsw_ctx *c, int sms) {
    if (!c || sms < 0) return set_err(GSW_EINVAL, "context or SM limit");
    c->sms = (sms == 0 || sms > c->sms_all) ? c->sms_all : sms;
    return GSW_OK;
}

int gsw_context_destroy(gsw_ctx *c) {
    if (!c) return GSW_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    DevBuf *all[] = {&c->plan_keys, &c->plan_order, &c->plan_small, &c->fill_cm, &c->fill_bnd, &c->trace_dirs,
                     &c->trace_ops, &c->band_scr, &c->misc, &c->io_q, &c->io_t, &c->io_qoff, &c->io_toff, &c->io_qlen,
                     &c->io_tlen, &c->io_res, &c->io_cigar, &c->io_colmax, &c->io_cmoff, &c->prof_qoff,
                     &c->prof_qlen, &c->ring_meta, &c->io_qp, &c->io_tp};
    c->st = nullptr;
    c->capturing = false;
    for (GraphCache &gc : c->seg)
        for (GraphSeg &g : gc.e)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    for (DevBuf *b : all) release(c, *b);
    cudaDeviceSynchronize();
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->host_small) cudaFreeHost(c->host_small);
    for (int k = 0; k <= GSW_NSTAGES; k++)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    destroy_aux(c->aux);
    delete c;
    return GSW_OK;
}

int gsw_align_batch(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                    const uint8_t *t, const int64_t *t_off, const int32_t *t_len, const int8_t *matrix,
                    int32_t alphabet, int32_t gap_open, int32_t gap_extend, uint32_t flags, int32_t mask_len,
                    gsw_result *results, uint32_t *cigar, int64_t cigar_capacity, int32_t *colmax,
                    const int64_t *colmax_off, void *stream) {
    Scoring sc;
    GSW_TRY(make_scoring(matrix, alphabet, gap_open, gap_extend, &sc));
    if ((flags & GSW_PACKED2) && alphabet != 4) return set_err(GSW_EINVAL, "GSW_PACKED2 needs the 4-letter alphabet");
    if (flags & GSW_PLAIN) return plain_impl(ctx, npairs, q, q_off, q_len, t, t_off, t_len, sc, flags,
                                                  mask_len, results, cigar, cigar_capacity, colmax, colmax_off,
                                                  (cudaStream_t)stream);
    return batch_impl(ctx, npairs, q, q_off, q_len, t, t_off, t_len, sc, flags, mask_len, results, cigar,
                      cigar_capacity, colmax, colmax_off, (cudaStream_t)stream);
}

int gsw_profile_create(gsw_ctx *ctx, const uint8_t *query, int32_t qlen, const int8_t *matrix, int32_t alphabet,
                       int32_t gap_open, int32_t gap_extend, gsw_profile **out) {
    if (!ctx || !out || (!query && qlen > 0) || qlen < 0 || qlen >= (1 << 24))
        return set_err(GSW_EINVAL, "bad profile arguments");
    *out = nullptr;
    Scoring sc;
    GSW_TRY(make_scoring(matrix, alphabet, gap_open, gap_extend, &sc));
    for (int32_t i = 0; i < qlen; i++)
        if (query[i] >= alphabet) return set_err(GSW_EINVAL, "query letter code %d >= alphabet", query[i]);
    CUDA_TRY(cudaSetDevice(ctx->device));
    gsw_profile *p = new (std::nothrow) gsw_profile();
    if (!p) return set_err(GSW_ENOMEM, "host allocation");
    p->ctx = ctx;
    p->qlen = qlen;
    p->sc = sc;
    cudaError_t e = cudaMalloc(&p->query, std::max(qlen, 1));
    if (e == cudaSuccess && qlen > 0) e = cudaMemcpy(p->query, query, qlen, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->query) cudaFree(p->query);
        delete p;
        return set_err(GSW_ENOMEM, "profile: %s", cudaGetErrorString(e));
    }
    *out = p;
    return GSW_OK;
}

int gsw_profile_destroy(gsw_profile *p) {
    if (!p) return GSW_OK;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(p->query);
    delete p;
    return GSW_OK;
}

int gsw_align_profile(gsw_ctx *ctx, const gsw_profile *prof, int32_t ntargets, const uint8_t *t,
                      const int64_t *t_off, const int32_t *t_len, uint32_t flags, int32_t mask_len,
                      gsw_result *results, uint32_t *cigar, int64_t cigar_capacity, int32_t *colmax,
                      const int64_t *colmax_off, void *stream) {
    if (!ctx || !prof || prof->ctx != ctx) return set_err(GSW_EINVAL, "bad profile or context");
    GSW_TRY(check_common(ctx, ntargets, flags));
    if (flags & GSW_PACKED2) return set_err(GSW_EINVAL, "GSW_PACKED2 is for gsw_align_batch");
    if (ntargets == 0) return GSW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (flags & GSW_HOST_IO) {
        std::vector<int64_t> qo(ntargets, 0);
        std::vector<int32_t> ql(ntargets, prof->qlen);
        std::vector<uint8_t> qh(std::max(prof->qlen, 1));
        if (prof->qlen) CUDA_TRY(cudaMemcpy(qh.data(), prof->query, prof->qlen, cudaMemcpyDeviceToHost));
        return batch_impl(ctx, ntargets, qh.data(), qo.data(), ql.data(), t, t_off, t_len, prof->sc, flags,
                          mask_len, results, cigar, cigar_capacity, colmax, colmax_off, st);
    }
    ctx->st = st;
    GSW_TRY(ensure(ctx, ctx->prof_qoff, sizeof(int64_t) * ntargets));
    GSW_TRY(ensure(ctx, ctx->prof_qlen, sizeof(int32_t) * ntargets));
    CUDA_TRY(launch_fill_const64((int64_t *)ctx->prof_qoff.p, 0, ntargets, st));
    CUDA_TRY(launch_fill_const((int32_t *)ctx->prof_qlen.p, prof->qlen, ntargets, st));
    return batch_impl(ctx, ntargets, prof->query, (const int64_t *)ctx->prof_qoff.p,
                      (const int32_t *)ctx->prof_qlen.p, t, t_off, t_len, prof->sc, flags, mask_len, results,
                      cigar, cigar_capacity, colmax, colmax_off, st);
}

}  // extern "C"
