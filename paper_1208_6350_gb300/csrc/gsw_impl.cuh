// Internal declarations shared by the library's translation units (device
// kernels and the host runtime behind include/gsw.h).  Nothing here is part of
// the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "gsw.h"

// Results owned by the library (gsw_align_batch_results, gsw_serve_poll_results):
// host copies of the records, the CIGAR words they index and, with GSW_COLMAX,
// the max arrays; released by gsw_results_free.
struct gsw_results {
    std::vector<gsw_result> res;
    std::vector<uint32_t> cigar;
    std::vector<int32_t> colmax;
    std::vector<int64_t> colmax_off;  // per pair, into colmax (empty without GSW_COLMAX)
    std::vector<int32_t> t_len;       // per pair
};

namespace gsw {

constexpr int kMaxAlpha = 32;

// Scoring scheme, passed by value to kernels (lives in the parameter bank).
struct Scoring {
    int32_t A;      // alphabet size
    int32_t O, X;   // gap open / extend, positive, O >= X: a gap of length k costs O + (k-1) X
    int32_t wmax;   // max matrix entry
    int32_t wmin;   // min matrix entry
    int32_t dna4;   // 1 when A == 4: the fill uses the letter-pair profile
    int32_t one;    // 1, unknown to the compiler: x * one + y issues as an integer multiply-add on the FMA pipe
    int8_t W[kMaxAlpha * kMaxAlpha];  // W[a * A + b]: query letter a vs target letter b
    int8_t fill_class[GSW_TUNE_BUCKETS];  // tuned 16-bit fill class per query-row bucket, -1: default rule
};

// Batch view (device pointers) shared by every stage.
struct BatchView {
    const uint8_t *q;
    const int64_t *q_off;
    const int32_t *q_len;
    const uint8_t *t;
    const int64_t *t_off;
    const int32_t *t_len;
    gsw_result *res;
    int32_t npairs;
    uint32_t flags;
    int32_t mask_len;  // < 0: max(m/2, 15)
    int32_t *colmax;
    const int64_t *colmax_off;
    uint32_t *cigar;
    int64_t cigar_cap;
    unsigned long long *cigar_cursor;
};

// Stage of the pipeline a fill launch serves.
enum FillMode : int32_t {
    kFillForward = 0,  // forward local fill: score1, ends, max array, secondary
    kFillRerun = 1,    // forward fill in 32-bit lanes for pairs whose 16-bit fill overflowed
    kFillReverse = 2,  // reversed fill from the end: begins (pairs whose reverse band is wide)
    kPlanBand = 3,     // not a fill: classes of the thread-per-pair band kernel
    kPlanTrace = 4,    // not a fill: pairs left to the warp traceback
};

// Kernel variants: (threads per pair P, row-words per thread R, 32-bit
// lanes).  A 16-bit variant covers 2*P*R query rows per strip, a 32-bit one
// P*R; longer queries run in several strips.  X(id, P, R, s32)
#define GSW_FILL_VARIANTS(X) \
    X(0, 16, 2, 0)           \
    X(1, 16, 3, 0)           \
    X(2, 16, 4, 0)           \
    X(3, 16, 5, 0)           \
    X(4, 16, 6, 0)           \
    X(5, 16, 7, 0)           \
    X(6, 16, 8, 0)           \
    X(7, 32, 8, 1)           \
    X(8, 8, 8, 0)            \
    X(9, 8, 10, 0)           \
    X(10, 8, 12, 0)          \
    X(11, 8, 14, 0)          \
    X(12, 8, 16, 0)
struct Variant {
    int P, R, s32;
};
constexpr int kNumVariants = 13;
constexpr int kVarS32 = 7;
constexpr int kVarMaxS16 = 6;  // the default rule picks among 0..6
// 8..12: one pair per 8 lanes with 8..16 row words per lane (128..256 rows per
// strip): twice the cells per lane and step of the 16-lane variants, so the
// per-step costs (shuffles, letter loads, trackers) weigh half as much; chosen
// per query length by the autotuner
constexpr int kVarP8First = 8;
// Two more fill classes: pairs whose query spans many strips run on a whole
// CTA (k_fill_long), one 32-lane warp per strip, strips pipelined across the
// CTA's warps; 16-bit lanes (2*32*16 = 1,024 rows per strip for DNA, 2*32*8 =
// 512 for general alphabets) or 32-bit lanes (256 rows per strip).  One pair
// per task.
constexpr int kClassLong16 = kNumVariants;
constexpr int kClassLong32 = kNumVariants + 1;
constexpr int kNumFillClasses = kNumVariants + 2;
__host__ __device__ inline Variant variant_at(int v) {
    switch (v) {
#define GSW_VARIANT_CASE(id, P, R, S32) \
    case id: return Variant{P, R, S32};
        GSW_FILL_VARIANTS(GSW_VARIANT_CASE)
#undef GSW_VARIANT_CASE
    case kClassLong16: return Variant{32, 16, 0};  // (DNA; general alphabets 8 row words)
    default: return Variant{32, 8, 1};
    }
}
// A query goes to the CTA kernel when it spans more than 3.5 x 512 rows of
// 4-letter DNA (a few such pairs in flight keep every warp busy), or more than
// 8 x 512 rows of a general alphabet (whose CTA holds fewer warps per SM).
__host__ __device__ inline bool long_pair(int rows, bool s32, bool dna) {
    const int sp = s32 ? 256 : 512;
    return dna ? 2 * rows > 7 * sp : rows > 8 * sp;
}
__host__ __device__ inline int variant_rows(int v) {
    Variant x = variant_at(v);
    return x.s32 ? x.P * x.R : 2 * x.P * x.R;
}

// The smallest one-strip 16-lane variant holding a query of `rows`, or the
// tallest (several strips).
__host__ __device__ inline int pick_s16(int rows) {
    for (int v = 0; v <= kVarMaxS16; v++)
        if (variant_rows(v) >= rows) return v;
    return kVarMaxS16;
}

// 16-bit fill class of a query of `rows` (>= 1): the tuned class of its
// bucket, else the smallest one-strip variant, or the CTA class for queries
// of many strips.
__host__ __device__ inline int pick_class16(int rows, const Scoring &sc) {
    const int b = (rows - 1) / GSW_TUNE_ROWS;
    if (rows >= 1 && b < GSW_TUNE_BUCKETS && sc.fill_class[b] >= 0) {
        const int c = sc.fill_class[b];  // public codes: 0..6, 8 CTA, 9..13 8-lane variants
        return c == 8 ? kClassLong16 : (c >= 9 ? kVarP8First + (c - 9) : c);
    }
    return long_pair(rows, false, sc.dna4) ? kClassLong16 : pick_s16(rows);
}

// Class of the reversed fill of a query whose end row is rows - 1 (plan.cu):
// the forward rule, or the 32-bit classes for a pair in 32-bit lanes; a DNA
// query of several strips reverses in the CTA kernel.
__host__ __device__ inline int pick_class_reverse(int rows, bool s32, const Scoring &sc) {
    int v = s32 ? (long_pair(rows, true, sc.dna4) ? kClassLong32 : kVarS32) : pick_class16(rows, sc);
    if (sc.dna4 && v != kClassLong16 && v != kClassLong32 && rows > variant_rows(v))
        v = v == kVarS32 ? kClassLong32 : kClassLong16;
    return v;
}

// The fill classes a launch of `mode` can meet when no query has more than
// maxm rows (a superset; each fill launch leaves the other classes out).
// force_s32: the batch runs in 32-bit lanes; s32: some pair may have been
// refilled in 32-bit lanes.  Empty pairs of the forward fill take class 0.
inline uint32_t fill_class_mask(int mode, int maxm, const Scoring &sc, bool force_s32, bool s32) {
    uint32_t m = 0;
    const int upto = maxm < GSW_TUNE_BUCKETS * GSW_TUNE_ROWS ? maxm : GSW_TUNE_BUCKETS * GSW_TUNE_ROWS;
    if (mode == kFillForward && force_s32) return (1u << kVarS32) | (1u << kClassLong32);
    if (mode == kFillRerun) return (1u << kVarS32) | (1u << kClassLong32);
    if (mode == kFillForward) m |= 1u << 0;
    for (int r = 1; r <= upto; r++) {
        if (mode == kFillForward) {
            m |= 1u << pick_class16(r, sc);
        } else {
            m |= 1u << pick_class_reverse(r, false, sc);
            if (s32) m |= 1u << pick_class_reverse(r, true, sc);
        }
    }
    if (maxm > upto) {  // past the tuned buckets: the tallest variant or the CTA classes
        m |= (1u << kVarMaxS16) | (1u << kClassLong16);
        if (s32 && mode != kFillForward) m |= (1u << kVarS32) | (1u << kClassLong32);
    }
    return m;
}

// Work plan of one fill launch: pairs sorted by (variant, cost descending),
// cut into warp tasks of 32/P pairs of one variant.  Task indices are handed
// out heaviest variant first (variant index descending).
struct FillPlan {
    const int32_t *order;      // sorted pair indices
    const int32_t *var_start;  // [kNumFillClasses+1] start of each class's pairs in `order`
    const int32_t *task_lo;    // [kNumFillClasses] first task index of each class
    const int32_t *task_hi;    // [kNumFillClasses] one past its last task index
    int32_t *head;             // [kNumFillClasses] task counters (zeroed by the plan)
    const int32_t *ntasks;     // total tasks
};

// Per-slot scratch of a persistent fill launch (one slot per pair in flight).
struct FillScratch {
    void *colmax;    // slots x ncap elements (uint16 biased for 16-bit, int32 for 32-bit)
    void *boundary;  // slots x 2 x ncap boundary words (uint32 for 16-bit, int2 for 32-bit)
    int32_t ncap;    // columns per slot (a multiple of 4: 8-byte stores of four 16-bit maxima)
    int32_t nslots;  // slots allocated
};

struct FillLaunch {
    BatchView b;
    Scoring sc;
    FillPlan plan;
    FillScratch scr;
    int32_t mode;
    uint32_t class_mask;  // classes launched (bit c: class c); the others hold no pair
    // nonzero once the batch's letter check found a code >= the alphabet
    // (written by the check, which runs first on the stream): the fill then
    // writes empty records and touches no letter, so its steady steps need
    // no clamp (the call returns GSW_EINVAL)
    const int32_t *bad_letters;
};

// internal per-pair bits (besides the public GSW_RES_*)
constexpr int32_t kResPendingS32 = 0x40;  // 16-bit fill overflowed: refill in 32-bit lanes
constexpr int32_t kResInternal = GSW_RES_INTERNAL;  // a consistency check failed (should never happen)
constexpr int32_t kResInvalid = GSW_RES_INVALID;    // gsw_fill_static: the pair's inputs were rejected
constexpr int32_t kResPendingTrace = 0x100;  // band too wide for one thread: warp traceback

// The thread-per-pair band kernel handles bands up to this many diagonals and
// this many rows; wider or longer pairs use the ring reverse fill and the warp
// traceback.
constexpr int kBandMaxWidth = 32;
constexpr int kBandMaxRows = 4096;
// Reverse bands the thread-per-pair kernel takes; wider ones reverse in the
// 16-bit ring fill (the begin), the CIGAR still comes from the band kernel
// when the traceback band is narrow.  (Measured with 16 on the short-read
// workload: band 8.26 -> 6.69 ms but ring reverse 1.89 -> 3.99 ms, so 32.)
constexpr int kBandMaxRevWidth = 32;

// Below this many pairs the thread-per-pair band kernel would occupy a few
// percent of the GPU's threads: the begins then come from the ring reverse
// fill and the CIGARs from the warp tracebacks.
constexpr int kSmallBatch = 1 << 14;
__host__ __device__ inline bool small_batch(const BatchView &b) { return b.npairs < kSmallBatch; }

constexpr int kPlanBinsPerVariant = 1024;
constexpr int kPlanBins = kNumFillClasses * kPlanBinsPerVariant;

// Width of the window the reversed fill scans, ending at the end column: an
// optimal alignment ending at (end_q, end_t) with score1 has at most
// D = ((end_q+1)*wmax - score1 - O)/X + 1 target letters against gaps (every
// gap run costs at least O + (len-1)X when O >= X), so it begins within
// end_q + 1 + D columns of the end.
__host__ __device__ inline int reverse_window(int end_q, int end_t, int score1, const Scoring &sc) {
    if (sc.X <= 0) return end_t + 1;
    long long d = (long long)(end_q + 1) * sc.wmax - score1 - sc.O;
    d = d < 0 ? 0 : d / sc.X + 1;
    long long w = (long long)end_q + 1 + d;
    long long lim = (long long)end_t + 1;
    return (int)(w < lim ? w : lim);
}

// Largest number of gap letters an alignment ending at (end_q, end_t) with
// score1 can hold: its at most end_q+1 aligned pairs score <= (end_q+1)*wmax,
// and g gap letters cost at least O + (g-1)X (O >= X).  -1 means unbounded.
__host__ __device__ inline int reverse_gap_bound(int end_q, int score1, const Scoring &sc) {
    long long num = (long long)(end_q + 1) * sc.wmax - score1 - sc.O;
    if (num < 0) return 0;
    if (sc.X <= 0) return -1;
    long long g = num / sc.X + 1;
    return g > (1 << 30) ? (1 << 30) : (int)g;
}

// Largest number of query letters against gaps it can hold: each also takes
// a row from the at most end_q+1 that could be aligned pairs, so g of them
// satisfy (end_q+1-g)*wmax - O - (g-1)X >= score1.  On the reversed
// sequences these are the steps below the main diagonal: the reverse band is
// [-reverse_gap_bound_rows, reverse_gap_bound], much narrower below.
__host__ __device__ inline int reverse_gap_bound_rows(int end_q, int score1, const Scoring &sc) {
    const long long num = (long long)(end_q + 1) * sc.wmax - score1 - sc.O + sc.X;
    const long long den = (long long)sc.wmax + sc.X;
    if (num < 0 || den <= 0) return 0;
    const long long g = num / den;
    return g > end_q + 1 ? end_q + 1 : (int)g;
}

// Diagonals of the reverse band: G above, reverse_gap_bound_rows below; -1
// when unbounded (extend 0)
__host__ __device__ inline int reverse_band_width(int end_q, int score1, const Scoring &sc) {
    const int G = reverse_gap_bound(end_q, score1, sc);
    if (G < 0) return -1;
    return G + reverse_gap_bound_rows(end_q, score1, sc) + 1;
}

// Half-width of the band of the global alignment between begin and end
// (la x lb letters, optimum score1): a path through diagonal d has at least
// g = |d| + |lb - la - d| gap letters and (la + lb - g)/2 aligned pairs, so
// scores at most wmax*floor((la+lb-g)/2) - O - (g-1)X; diagonals where that
// bound is below score1 carry no optimal path.  Returns w such that the band
// is [min(0, lb-la) - w, max(0, lb-la) + w].
__host__ __device__ inline int band_halfwidth(int la, int lb, int score1, const Scoring &sc) {
    const int delta = lb - la;
    const int g0 = delta < 0 ? -delta : delta;
    auto ub = [&](long long g) -> long long {
        long long aligned = ((long long)la + lb - g) / 2;
        long long s = (long long)sc.wmax * aligned;
        if (g > 0) s -= sc.O + (g - 1) * (long long)sc.X;
        return s;
    };
    // largest w with ub(g0 + 2w) >= score1 (ub is non-increasing in g)
    int lo = 0, hi = la + lb + 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (ub(g0 + 2LL * mid) >= score1) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Diagonal range [dlo, dhi] of the traceback band, clipped to the rectangle.
__host__ __device__ inline int band_range(int la, int lb, int score1, const Scoring &sc, int *dlo, int *dhi) {
    const int w = band_halfwidth(la, lb, score1, sc);
    const int delta = lb - la;
    int lo = (delta < 0 ? delta : 0) - w, hi = (delta > 0 ? delta : 0) + w;
    lo = lo < -la ? -la : lo;
    hi = hi > lb ? lb : hi;
    *dlo = lo;
    *dhi = hi;
    return hi - lo + 1;
}

// Traceback classes of the pairs the band kernel leaves (bands wider than 32
// diagonals, or small batches): 0-3 anti-diagonal warp kernel (bands of at
// most 64/128/256/512 diagonals), 4 the CTA strip kernel (wider bands), 5-8
// the 16-bit full-rectangle kernel with strips of 64/128/192/256 query rows
// (8 lanes x R = 4/8/12/16 words x 2 halves; regions taller than the class's
// strip run several strips: 256-row strips for DNA; other alphabets 64-row
// strips, and 128-row ones with a larger scratch allowance for regions whose
// decisions exceed kT16MaxWords in 64-row strips).
#ifndef GSW_T16_GEN_VMAX
#define GSW_T16_GEN_VMAX 0
#endif
constexpr int kTraceRingClass = 4;
constexpr int kTraceT16First = 5;
constexpr int kTraceT16Classes = 4;
constexpr int kT16P = 8;                   // lanes per pair
constexpr int kT16MaxCols = 4096;          // longest target region of the 16-bit kernel
constexpr long long kT16MaxWords = 1 << 17;  // scratch words of one pair (512 KB)
// general alphabets: regions over kT16MaxWords in 64-row strips take the
// 128-row class with this allowance (its own launch and scratch, so the few
// large pairs do not shrink the groups of the others)
constexpr long long kT16MaxWordsBig = 1 << 20;
__host__ __device__ inline int t16_R(int v) { return 4 * (v + 1); }
__host__ __device__ inline int t16_strip_rows(int v) { return 2 * kT16P * t16_R(v); }
__host__ __device__ inline int t16_strips(int la, int v) { return (la + t16_strip_rows(v) - 1) / t16_strip_rows(v); }
__host__ __device__ inline int t16_steps(int lb) { return lb + 2 * kT16P - 1; }
// direction words of one pair (strips x steps x R/4 words x 8 lanes)
__host__ __device__ inline long long t16_dir_words(int la, int lb, int v) {
    return (long long)t16_strips(la, v) * t16_steps(lb) * (t16_R(v) / 4) * kT16P;
}
// scratch words of one pair: direction words, then two boundary rows (one
// word per column) when it has several strips
__host__ __device__ inline long long t16_need_words(int la, int lb, int v) {
    const long long d = t16_dir_words(la, lb, v);
    return t16_strips(la, v) > 1 ? d + 2LL * ((lb + 3) & ~3) : d;
}
// small: a batch of fewer than 2^14 pairs (the rectangle needs a wider margin
// there, where the anti-diagonal kernel's one pair per warp keeps more pairs
// in flight)
__host__ __device__ inline int trace_class(int la, int lb, int score1, const Scoring &sc, bool small, int *dlo,
                                           int *dhi) {
    const int width = band_range(la, lb, score1, sc, dlo, dhi);
    const int ad = width <= 64 ? 0 : width <= 128 ? 1 : width <= 256 ? 2 : width <= 512 ? 3 : kTraceRingClass;
    if (la >= 1 && lb >= 1 && lb <= kT16MaxCols) {
        // general alphabets keep A x R profile words per lane: 64-row strips
        // (128 measured 2.5 % slower on protein search: a third of the warps per SM)
        const int vmax = sc.dna4 ? kTraceT16Classes - 1 : GSW_T16_GEN_VMAX;
        const int v0 = (la - 1) / 64;
        int v = v0 < vmax ? v0 : vmax;
        long long cap = kT16MaxWords;
        if (!sc.dna4 && v == 0 && t16_need_words(la, lb, 0) > kT16MaxWords) {
            v = 1;
            cap = kT16MaxWordsBig;
        }
        const long long rows = (long long)t16_strips(la, v) * t16_strip_rows(v);
        const long long cols = lb + 2 * kT16P;
        // every value of the DP over the padded rectangle lies in
        // [-(3O + X(rows + cols) + |wmin|), wmax * min(rows, cols) + wmax]:
        // it must fit a biased 16-bit lane
        const long long lo = 3LL * sc.O + (long long)sc.X * (rows + cols + 2) - (sc.wmin < 0 ? sc.wmin : 0);
        const long long hi = (long long)sc.wmax * ((cols < rows ? cols : rows) + 1);
        if (lo <= 30000 && hi <= 30000 && t16_need_words(la, lb, v) <= cap) {
            // cell updates: the padded rectangle against the band's
            // anti-diagonal slots; a 16-bit pair of cells costs about the
            // instructions of one 32-bit anti-diagonal cell
            // (bands wider than 512 diagonals: the rectangle always)
            const long long rect = rows * t16_steps(lb);
            if (ad == kTraceRingClass) return kTraceT16First + v;
            const long long band = (32LL << ad) * (la + lb + 1);
            if (rect <= (small ? 2 : 3) * band) return kTraceT16First + v;
        }
    }
    return ad;
}

// stage launchers (host side, enqueue on `st`)
// Status of a completed batch from what its kernels counted, in order of
// precedence: letter codes outside the alphabet (GSW_EINVAL), records that
// failed a consistency check (GSW_EINTERNAL), CIGAR words beyond the
// caller's capacity (GSW_ECIGAR_SPACE, only with GSW_CIGAR).
__host__ __device__ inline int batch_status(int bad_letters, unsigned long long internal, bool cigar,
                                            unsigned long long cigar_words, long long cigar_capacity) {
    if (bad_letters) return GSW_EINVAL;
    if (internal) return GSW_EINTERNAL;
    if (cigar && cigar_words > (unsigned long long)(cigar_capacity < 0 ? 0 : cigar_capacity)) return GSW_ECIGAR_SPACE;
    return GSW_OK;
}

// Host helpers of the runtime (api.cu): the calling thread's error detail,
// the scoring checks shared by every entry point, and the count of records
// flagged kResInternal (one small kernel and a readback on `st`).
int set_err(int code, const char *fmt, ...);
int make_scoring(const int8_t *matrix, int32_t A, int32_t O, int32_t X, Scoring *sc);
cudaError_t launch_count_flag(const gsw_result *res, int32_t n, int32_t flag, unsigned long long *count,
                              cudaStream_t st);

int fill_block_threads();
// largest number of slots (pairs in flight) of any variant's launch
int fill_slots(const Scoring &sc, int sms);
// Largest number of pairs a warp of a fill variant holds at once (32 / P for
// the narrowest group): the slots a capped launch needs per warp.
int fill_max_pairs_per_warp();
// one persistent launch per class in fl.class_mask, heaviest first; each grid
// capped at max_blocks and at the slots the scratch holds
cudaError_t launch_fill(const FillLaunch &fl, int sms, int max_blocks, cudaStream_t st);

struct PlanBuffers {
    int32_t *keys;       // [npairs]
    int32_t *hist;       // [kPlanBins]
    int32_t *binoff;     // [kPlanBins]
    int32_t *cursor;     // [kPlanBins]
    int32_t *order;      // [npairs]
    int32_t *var_start;  // [kNumFillClasses+1]
    int32_t *task_lo;    // [kNumFillClasses]
    int32_t *task_hi;    // [kNumFillClasses]
    int32_t *ntasks;     // [1]
    int32_t *head;       // [kNumFillClasses]
};
cudaError_t launch_plan(const BatchView &b, const Scoring &sc, int32_t mode, const PlanBuffers &pb,
                        cudaStream_t st);

// Wide-band traceback (trace_ring.cu): banded global fill with direction
// bits on the CTA strip pipeline, then a warp walk per pair, group by group
// of pairs whose direction words fit the pool.
struct RingLaunchArgs {
    BatchView b;
    Scoring sc;
    const int32_t *order;     // plan order
    const int32_t *var_start; // class boundaries in `order`
    const long long *prefix;  // [n + 1] from launch_ring_needs
    int *final_h;             // [n]
    int *group;               // 3 ints: g0 (zeroed by the caller before the first group), g1, head
    uint32_t *pool;
    long long pool_words;
    int2 *bnd;                // boundary buffers: slots x bnd_stride int2
    long long bnd_stride;
    int slots;
    uint32_t *ops;            // walk: walk_warps x op_words
    long long op_words;
    int walk_warps;
};
int ring_trace_class();
int context_device(const gsw_ctx *ctx);
// Rounds a call's shapes (largest lengths, traceback scratch) up to powers of
// two, so that calls of similar shape repeat a captured pipeline (serving).
void context_set_graph_buckets(gsw_ctx *ctx, bool on);
int ring_slots_per_cta();
// prefix sums of the class's direction words; out[0] total, [1] max words of a pair, [2] max op words
cudaError_t launch_ring_needs(const BatchView &b, const Scoring &sc, const int32_t *order, const int32_t *var_start,
                              long long *prefix, unsigned long long *out, cudaStream_t st);
cudaError_t launch_ring_group(const RingLaunchArgs &a, int sms, cudaStream_t st);

struct TraceScratch {
    uint32_t *dirs;         // per warp: dir_words words (global direction bit-planes)
    int64_t dir_words;      // per warp
    uint32_t *ops;          // per warp: op_words words (reversed CIGAR runs)
    int64_t op_words;       // per warp
    const int32_t *order;   // pairs to trace: order[var_start[0] .. var_start[1])
    const int32_t *var_start;
};
int trace_block_threads();
// largest needs of a pair: [0] direction words of the anti-diagonal classes,
// [1] op words of the warp classes; need16[v]: direction words of 16-bit class v
cudaError_t launch_trace_need(const BatchView &b, const Scoring &sc, unsigned long long *max_need,
                              unsigned long long *need16, cudaStream_t st);
cudaError_t launch_trace_ad(const BatchView &b, const Scoring &sc, const TraceScratch &ts, int grid,
                            cudaStream_t st);

// 16-bit full-rectangle traceback (trace16.cu): per class v (strips of
// 64(v+1) rows) and group of 8 lanes, dir_words[v] direction words (0: no
// pairs) and op_words op words; the classes run one after the other on the
// stream and share the buffers
struct T16Scratch {
    uint32_t *dirs;
    int64_t dir_words[kTraceT16Classes];  // per group
    uint32_t *ops;
    int64_t op_words;   // per group
    const int32_t *order;
    const int32_t *var_start;
    int32_t *head;      // per-class task counters (zeroed by the plan)
    int warps[kTraceT16Classes];  // warps of each class's launch (the scratch holds 4 groups each)
};
// warps of class v's launch that can be resident
int t16_max_warps(const Scoring &sc, int sms, int v);
cudaError_t launch_trace16(const BatchView &b, const Scoring &sc, const T16Scratch &ts, int sms, cudaStream_t st);

int band_block_threads();
// Grids and scratch of the three band classes (widths 8, 16, 32), each
// sized to the blocks that can be resident, scaled down to the budget.
struct BandGrids {
    int grid[3];
    int64_t words[3];  // per warp
    size_t off[3];     // byte offsets of the classes' scratch
    size_t total_bytes;
};
BandGrids band_grids(int rows_cap, int sms, size_t budget_bytes);
struct BandStreams {
    cudaStream_t s[2];
    cudaEvent_t fork, join[2];
};
cudaError_t launch_band(const BatchView &b, const Scoring &sc, const PlanBuffers &pb, void *scratch,
                        const BandGrids &g, cudaStream_t st, const BandStreams &aux);

// small helpers (misc.cu)
// one pass over the pairs: [0, 1] largest lengths, [2, 3] arena extents,
// [4] nonzero if a length is outside [0, 2^24) or an offset negative
cudaError_t launch_batch_stats(const int64_t *q_off, const int32_t *q_len, const int64_t *t_off,
                               const int32_t *t_len, int32_t n, unsigned long long *out5, cudaStream_t st);
// 2-bit packed DNA letters to one byte per letter
cudaError_t launch_unpack2(const uint8_t *in, uint8_t *out, long long nletters, cudaStream_t st);
cudaError_t launch_validate(const BatchView &b, const Scoring &sc, int32_t *bad, cudaStream_t st);
cudaError_t launch_fill_const(int32_t *dst, int32_t v, int32_t n, cudaStream_t st);
cudaError_t launch_fill_const64(int64_t *dst, int64_t v, int32_t n, cudaStream_t st);

}  // namespace gsw
