/*
 * gsw.h -- C ABI of the GB300 (sm_103a) SSW alignment library.
 *
 * The library computes, for each (query, target) pair, what the SSW paper
 * (Zhao, Lee, Garrison, Marth 2012) describes in "Algorithm and
 * implementation" and "Results / Usage": the optimal local Smith-Waterman-Gotoh
 * score, its end on target and query (found from the per-column "max" array
 * and the column that holds the matrix maximum), the suboptimal score from the
 * max array with the primary's neighbourhood masked, the begin by a reversed
 * SW from the end, and the alignment (CIGAR) by a banded SW between begin and
 * end.  All of it runs in this library's CUDA kernels; there is no CPU path.
 *
 * Conventions shared by every call:
 *   - Sequences are letter codes, one byte per residue, in [0, alphabet).
 *     A query of length m has rows i = 0..m-1; a target of length n has
 *     columns j = 0..n-1.  Positions in results are 0-based and inclusive.
 *   - matrix is alphabet x alphabet int8, row-major, matrix[a*alphabet + b] =
 *     score of query letter a against target letter b (host memory, copied).
 *   - gap_open O and gap_extend X are non-negative with O >= X; a gap of
 *     length k costs O + (k-1)*X (the paper prints penalties, e.g. "gap open
 *     -2 and extension -1" in the Fig. 1 caption, without fixing this
 *     convention; this is the reading the library implements).
 *   - Ties: the end is the first target column whose max equals the optimum,
 *     then the first query row in that column with it; the begin is the
 *     largest (target, query) begin among optimal alignments ending there; the
 *     CIGAR is the one traced back from the end preferring a match/mismatch
 *     column, then a target gap (D), then a query gap (I), and closing a gap as
 *     early as possible.
 *   - Errors: every call returns GSW_OK (0) or a negative GSW_E* code and
 *     never throws; gsw_strerror() names the code, gsw_last_error() gives a
 *     one-line detail for the calling thread.
 */
#ifndef GSW_H
#define GSW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSW_OK 0
#define GSW_EINVAL (-1)       /* bad argument (sizes, codes, scoring, flags) */
#define GSW_ENOMEM (-2)       /* device or pinned memory exhausted / over budget */
#define GSW_ECUDA (-3)        /* a CUDA runtime call failed */
#define GSW_ETIMEDOUT (-4)    /* a bounded wait gave up (serving loop) */
#define GSW_ECIGAR_SPACE (-5) /* the caller's CIGAR buffer is too small */
#define GSW_EOVERFLOW (-6)    /* a score does not fit in int32 arithmetic */
#define GSW_ENOTFOUND (-7)    /* unknown request id */
#define GSW_ESTATE (-8)       /* call not valid in the object's current state */
#define GSW_EINTERNAL (-9)    /* a pair failed one of the library's own consistency
                                 checks (a bug, never expected): its record carries
                                 GSW_RES_INTERNAL, every other record is complete */

/* flags for gsw_align_batch / gsw_align_profile */
#define GSW_BEGIN 0x1u      /* also run the reversed SW: ref_begin1, read_begin1 */
#define GSW_CIGAR 0x2u      /* also run the banded SW + traceback (implies GSW_BEGIN) */
#define GSW_COLMAX 0x4u     /* write the per-column max array to `colmax` */
#define GSW_HOST_IO 0x8u    /* every pointer argument is host memory; the call
                               stages it through the context and returns when
                               the results are back in host memory */
#define GSW_FORCE_S32 0x10u /* skip the 16-bit lanes (32-bit fill for every pair) */
#define GSW_PLAIN 0x20u     /* baseline: one fill/reverse/traceback launch
                               sequence per pair, no batching */
#define GSW_TIMING 0x40u    /* record CUDA events around each stage of the call
                               (read them with gsw_last_stats) */
#define GSW_PACKED2 0x80u   /* q and t are 2-bit packed DNA arenas: letter x (codes
                               0..3) in bits 2(x%4)..2(x%4)+1 of byte x/4; offsets
                               and lengths count letters; alphabet must be 4.  The
                               call expands them on the device (one kernel); not
                               with GSW_PLAIN or gsw_align_profile */

/* CIGAR words: (run_length << 4) | op, op 0 = M (match or mismatch column),
 * 1 = I (query letter against a gap), 2 = D (target letter against a gap). */
#define GSW_CIGAR_M 0u
#define GSW_CIGAR_I 1u
#define GSW_CIGAR_D 2u

/* per-pair status bits in gsw_result.flags */
#define GSW_RES_S32 0x1u          /* the fill ran in 32-bit lanes (16-bit overflowed or forced) */
#define GSW_RES_CIGAR_SPACE 0x2u  /* no room for this pair's CIGAR: cigar_len = -needed */
#define GSW_RES_INVALID 0x4u      /* gsw_fill_static only: the pair's lengths, offsets or
                                     letters were rejected; the record is the empty one */
#define GSW_RES_INTERNAL 0x80u    /* a consistency check of the kernels failed for this
                                     pair (the reversed maximum differs from score1, the
                                     traceback left its band, ...); the call returns
                                     GSW_EINTERNAL and the pair's begins / CIGAR are
                                     not to be trusted */

/*
 * One pair's result (Results, Usage: the record the paper lists for a call --
 * the optimum's score, where it lies and how it aligns, and the second-best
 * score with where it ends).  Missing values are -1: with score1 = 0 there is no
 * alignment and every position is -1; begins are -1 unless GSW_BEGIN or
 * GSW_CIGAR was given; score2 = 0 gives ref_end2 = -1.
 */
typedef struct gsw_result {
    int32_t score1;      /* optimal local score (>= 0) */
    int32_t score2;      /* largest max-array entry outside [ref_end1-L, ref_end1+L] */
    int32_t ref_begin1;  /* target begin of the optimal alignment */
    int32_t ref_end1;    /* target end: first column whose max equals score1 */
    int32_t read_begin1; /* query begin */
    int32_t read_end1;   /* query end: first row of column ref_end1 holding score1 */
    int32_t ref_end2;    /* first column holding score2 */
    int32_t cigar_len;   /* number of CIGAR words; 0 if none; -needed on GSW_RES_CIGAR_SPACE */
    int64_t cigar_off;   /* index of the first CIGAR word in the caller's buffer, -1 if none */
    int32_t flags;       /* GSW_RES_* bits */
    int32_t reserved;
} gsw_result;

typedef struct gsw_ctx gsw_ctx;
typedef struct gsw_profile gsw_profile;

/*
 * Creates a context on CUDA device `device`.  The context owns the device
 * scratch (work queues, per-slot column-max and strip-boundary buffers,
 * traceback scratch) and pinned staging for GSW_HOST_IO; it never holds more
 * than `mem_budget_bytes` of device memory (0 = 4 GiB); when a batch's
 * per-slot scratch would exceed it, fewer pairs run at a time.  One context
 * may be used by one host thread at a time.  Errors: GSW_EINVAL (bad
 * device), GSW_ECUDA, GSW_ENOMEM.
 * Paper: none (a GPU resource holder; the paper's library keeps no state
 * between calls beyond the query profile).
 */
int gsw_context_create(int device, size_t mem_budget_bytes, gsw_ctx **out);

/* Releases everything the context owns.  Waits for its work to finish. */
int gsw_context_destroy(gsw_ctx *ctx);

/*
 * Autotuner for the forward and reversed fills (16-bit lanes).  Queries are
 * bucketed by length in GSW_TUNE_ROWS-row buckets; for each bucket a fill class
 * is chosen: 0..6 = one pair per 16-lane group with 2..8 row words per lane
 * (64..256 query rows per strip; longer queries run several strips), 8 = one
 * pair per CTA (512-row strips pipelined across the warps), 9..13 = one pair
 * per 8-lane group with 8, 10, 12, 14, 16 row words per lane (128..256 rows
 * per strip), -1 = the default rule (the smallest one-strip class of 0..6, the
 * CTA class from 1792 rows).  The choice changes speed only: every class
 * gives the same results.
 * Paper: none for the tuner itself; it chooses among layouts of the one
 * fill the paper describes (Algorithm and implementation, item (1)).
 */
#define GSW_TUNE_BUCKETS 32
#define GSW_TUNE_ROWS 32
typedef struct gsw_tune {
    int8_t fill_class[GSW_TUNE_BUCKETS]; /* bucket b: queries of 32b+1 .. 32(b+1) rows */
    float gcups[GSW_TUNE_BUCKETS];       /* measured forward-fill rate of the chosen class */
    float gcups_default[GSW_TUNE_BUCKETS]; /* ... of the default rule's class */
} gsw_tune;

/* Measures every candidate class of every bucket on seeded random pairs
 * (queries of the bucket's largest length against targets of target_len
 * letters, the given scoring, score-only batches of about 2 G cells, best of 3
 * runs), installs the fastest in the context and copies the table to *out (may
 * be NULL).  Takes a few seconds; allocates its own temporary device buffers.
 * Errors: GSW_EINVAL, GSW_ENOMEM, GSW_ECUDA. */
int gsw_autotune(gsw_ctx *ctx, const int8_t *matrix, int32_t alphabet, int32_t gap_open, int32_t gap_extend,
                 int32_t target_len, gsw_tune *out);

/* Installs a table (e.g. one saved from gsw_autotune); NULL restores the
 * default rule.  Errors: GSW_EINVAL (a class outside -1..6, 8..13). */
int gsw_context_set_tune(gsw_ctx *ctx, const gsw_tune *tune);

/*
 * Reads against one long reference (whole viral, bacterial or chromosome
 * sequences; the paper's genome alignments, Results).  Every read gets the
 * record gsw_align_batch would give for the pair (read, whole reference):
 * score1, ends, score2 / ref_end2 over the whole reference's max array,
 * begins and CIGAR (flags GSW_BEGIN, GSW_CIGAR), bit-exact.  The reference is
 * cut into windows owning `window` columns (0: the default, at least 65,536)
 * that start earlier by the longest reference span of a positive-scoring
 * local alignment of the longest read, so the work is one batch of
 * reads x windows plus two small passes.  Pointers follow gsw_align_batch's
 * rules (GSW_HOST_IO: all host); ref_len < 2^31; the reads' lengths < 2^24.
 * Work and the read-back of device read lengths are ordered on `stream`, so
 * inputs written by work queued there before the call are seen.
 * Errors: GSW_EINVAL (arguments, or `window` smaller than 2 x mask + overlap),
 * GSW_ENOMEM, GSW_ECUDA, GSW_ECIGAR_SPACE (records complete, CIGARs that do
 * not fit have cigar_len = -needed).
 * Paper: Results (Performance: reads aligned against whole viral, bacterial
 * and chromosome sequences with the library).
 */
int gsw_align_to_reference(gsw_ctx *ctx, int32_t nreads, const uint8_t *q, const int64_t *q_off,
                           const int32_t *q_len, const uint8_t *ref, int64_t ref_len,
                           const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                           int32_t gap_extend, uint32_t flags, int32_t mask_len, int64_t window,
                           gsw_result *results, uint32_t *cigar, int64_t cigar_capacity,
                           void *stream);

/*
 * All-vs-all: every pair (i, j), i < j, of n sequences (the paper's read
 * overlaps, Applications), query = sequence i, target = sequence j; record k
 * is the pair of row-major triangle order, k = i*n - i*(i+1)/2 + (j - i - 1),
 * so results has n(n-1)/2 records (n <= 65,536).  Flags: GSW_BEGIN, GSW_CIGAR,
 * GSW_HOST_IO, GSW_PACKED2 as for gsw_align_batch; 0 = score only (score1,
 * ends, score2).  The pairs are generated on the device and run in chunks of
 * `chunk` pairs (0: 2^22) through the batched path; CIGAR offsets refer to the
 * whole `cigar` buffer.  Errors as gsw_align_batch.
 * Paper: Applications (the read-overlap use of the library).
 */
int gsw_align_all_pairs(gsw_ctx *ctx, int32_t n, const uint8_t *seq, const int64_t *off,
                        const int32_t *len, const int8_t *matrix, int32_t alphabet,
                        int32_t gap_open, int32_t gap_extend, uint32_t flags, int32_t mask_len,
                        int64_t chunk, gsw_result *results, uint32_t *cigar,
                        int64_t cigar_capacity, void *stream);

/* Sizes the context's persistent launches for at most `sms` SMs (0: all), so
 * that work of other streams finds free SMs while this context's kernels
 * run.  Results do not depend on it.  Errors: GSW_EINVAL (sms < 0). */
/* Paper: none (GPU scheduling). */
int gsw_context_set_sm_limit(gsw_ctx *ctx, int sms);

/*
 * Aligns npairs pairs: query p is q[q_off[p] .. q_off[p]+q_len[p]), target p
 * is t[t_off[p] .. t_off[p]+t_len[p]).  Lengths may be 0 (score1 = 0).
 *
 * Memory: q, q_off, q_len, t, t_off, t_len, results, cigar, colmax and
 * colmax_off are device pointers, unless flags has GSW_HOST_IO, in which case
 * they are all host pointers.  The caller owns every buffer.  `results` has
 * npairs records.  `cigar` has `cigar_capacity` uint32 words shared by the
 * batch (may be NULL with capacity 0 when GSW_CIGAR is not set); pairs that
 * do not fit are marked GSW_RES_CIGAR_SPACE and the call returns
 * GSW_ECIGAR_SPACE after filling everything else.  With GSW_COLMAX, colmax
 * receives t_len[p] int32 values at colmax[colmax_off[p]]; words outside
 * every pair's range are left unchanged.  With GSW_HOST_IO a negative
 * colmax_off is rejected (GSW_EINVAL); device offsets are the caller's to keep
 * inside its buffer.
 *
 * mask_len is the half-width L of the window masked around ref_end1 before
 * the suboptimal score is taken; negative means max(q_len/2, 15).
 *
 * Stream: work is queued on `stream` (a cudaStream_t; NULL = the legacy
 * default stream).  The call reads a few values back from the device on that
 * stream (the longest query and target, the traceback scratch size, the CIGAR
 * words used), so it returns only when the batch's results are complete.
 *
 * Errors: GSW_EINVAL (alphabet not in [1, 32], matrix entries outside
 * [-127, 127], O < X, O or X > 255 or negative, npairs < 0, mask_len too
 * large), GSW_ENOMEM, GSW_ECUDA, GSW_ECIGAR_SPACE, GSW_EOVERFLOW (a pair whose
 * score or intermediate value exceeds int32 range cannot happen for lengths
 * below 2^24 and |W| <= 127; longer inputs are rejected with GSW_EINVAL).
 * GSW_EINTERNAL: a pair failed one of the kernels' own consistency checks
 * (never expected; its record carries GSW_RES_INTERNAL, the others are
 * complete).
 *
 * Paper: Algorithm and implementation, item (1) (the fill with the max array
 * and the recorded column, then the reversed SW for the begin and the banded
 * SW for the alignment) and item (2) (the suboptimal score from the masked
 * max array); Results, Usage (the record returned per alignment).
 */
int gsw_align_batch(gsw_ctx *ctx, int32_t npairs,
                    const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                    const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                    const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                    int32_t gap_extend, uint32_t flags, int32_t mask_len,
                    gsw_result *results, uint32_t *cigar, int64_t cigar_capacity,
                    int32_t *colmax, const int64_t *colmax_off, void *stream);

/*
 * Library-owned results.  The paper's library returns, for each alignment, a
 * record it allocates and the caller releases (Results, Usage: the optimum's
 * score, ends and begins, its traceback, and the second-best score with its
 * end).  gsw_align_batch_results runs gsw_align_batch on the same arguments
 * (GSW_HOST_IO decides whether the inputs are host or device memory; flags
 * and errors as gsw_align_batch, except that a CIGAR buffer is never too
 * small: the library reserves a sixteenth of each pair's shorter sequence
 * plus 4 words, and aligns the pairs whose CIGARs did not fit once more on
 * their own with the room they reported) and returns the records, CIGAR words and
 * (GSW_COLMAX) max arrays as one handle in host memory.  gsw_results_get
 * copies record i out as a gsw_record whose pointers point into the handle;
 * they stay valid until gsw_results_free.  On GSW_EINTERNAL the handle is
 * still returned (the flagged records carry GSW_RES_INTERNAL); on any other
 * error *out is NULL.  The call returns when the results are on the host.
 */
typedef struct gsw_results gsw_results;
typedef struct gsw_record {
    int32_t score1, score2;         /* optimal and suboptimal scores */
    int32_t ref_begin1, ref_end1;   /* target begin / end of the optimum (-1 if none) */
    int32_t read_begin1, read_end1; /* query begin / end of the optimum (-1 if none) */
    int32_t ref_end2;               /* target end of the suboptimal score (-1 if none) */
    uint8_t lane_bits_used;         /* 16 or 32: width of the fill lanes that gave score1 */
    const uint32_t *cigar;          /* cigar_len CIGAR words (GSW_CIGAR), else NULL */
    int32_t cigar_len;
    const int32_t *colmax;          /* n max-array values (GSW_COLMAX), else NULL */
    int32_t n;                      /* target length */
    int32_t flags;                  /* GSW_RES_* bits */
} gsw_record;

int gsw_align_batch_results(gsw_ctx *ctx, int32_t npairs, const uint8_t *q, const int64_t *q_off,
                            const int32_t *q_len, const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                            const int8_t *matrix, int32_t alphabet, int32_t gap_open, int32_t gap_extend,
                            uint32_t flags, int32_t mask_len, void *stream, gsw_results **out);
/* Records in the handle (0 for NULL). */
int32_t gsw_results_count(const gsw_results *res);
/* Copies record i (0 <= i < count) to *rec.  Errors: GSW_EINVAL. */
int gsw_results_get(const gsw_results *res, int32_t i, gsw_record *rec);
/* Releases the handle and everything its records point to (NULL is ignored). */
void gsw_results_free(gsw_results *res);

/*
 * ssw_init-style query profile: copies one query and its scoring onto the
 * device, where it stays until gsw_profile_destroy.  query is host memory.
 * Errors: as gsw_align_batch for the scoring arguments; GSW_ENOMEM.
 * Paper: Algorithm and implementation (the query profile is built once per
 * query and reused for every target, after Farrar).
 */
int gsw_profile_create(gsw_ctx *ctx, const uint8_t *query, int32_t qlen,
                       const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                       int32_t gap_extend, gsw_profile **out);
int gsw_profile_destroy(gsw_profile *prof);

/*
 * Aligns the profile's query against ntargets targets (layout and memory
 * rules of gsw_align_batch's t, t_off, t_len, results, cigar, colmax).
 * Paper: Results, Usage (one query aligned against many targets with one
 * profile).
 */
int gsw_align_profile(gsw_ctx *ctx, const gsw_profile *prof, int32_t ntargets,
                      const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                      uint32_t flags, int32_t mask_len, gsw_result *results,
                      uint32_t *cigar, int64_t cigar_capacity, int32_t *colmax,
                      const int64_t *colmax_off, void *stream);

/*
 * Statistics of the last gsw_align_batch / gsw_align_profile call on a
 * context.  kernel_launches counts the kernels the call enqueued.  With
 * GSW_TIMING, stage_ms holds CUDA-event times measured on the call's stream:
 *   [0] forward plan (device counting sort into warp tasks)
 *   [1] forward fill kernel (16-bit lanes, or 32-bit with GSW_FORCE_S32)
 *   [2] 32-bit refill of overflowed pairs (plan + kernel)
 *   [3] reversed fill in the ring kernel, for pairs whose reverse band is
 *       wider than 32 diagonals (plan + kernel)
 *   [4] thread-per-pair banded reverse and traceback (plan + kernels)
 *   [5] warp traceback of pairs whose traceback band is wider than 32
 *   [6] whole device pipeline ([0] .. [5])
 * Stages that did not run read 0.  The call has already waited for its work,
 * so reading the stats does not block.  graph_segments: how many of the two
 * pipeline segments (before / after the traceback readback) ran as a replay
 * of a captured CUDA graph: a call repeated with the same buffers, sizes,
 * flags and scoring on a non-default stream is captured on its second run and
 * replayed from the third.  Errors: GSW_EINVAL (NULL).
 * Paper: none (measurement).
 */
#define GSW_NSTAGES 7
typedef struct gsw_stats {
    int32_t kernel_launches;
    int32_t timed;
    float stage_ms[8];
    int32_t graph_segments;
    int64_t cigar_words;  /* CIGAR words the call needed (all pairs) */
    /* wide-band traceback (bands over 512 diagonals): direction words of all
     * its pairs, the pool they are written to, and the groups of pairs the
     * pool was used in one after the other (ring_words > ring_pool_words
     * means at least two groups held pairs) */
    int64_t ring_words, ring_pool_words;
    int32_t ring_groups;
    int32_t internal_pairs;  /* records flagged GSW_RES_INTERNAL */
} gsw_stats;
int gsw_last_stats(const gsw_ctx *ctx, gsw_stats *out);

/*
 * Allocation-free forward fill.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory -- code running where
 * cudaMalloc is forbidden or unsafe (a memory pool or arena owned by another
 * framework, a hard real-time loop that must not block on the allocator, or a
 * process whose device memory was reserved up front by a framework).  It must
 * not be called from a CUDA stream callback (cudaLaunchHostFunc): it issues
 * CUDA calls and waits for its stream.  It needs no context and allocates
 * nothing: the caller passes inputs and outputs, and the scratch of the pairs
 * in flight (their column maxima and strip boundaries) lives in one
 * file-scope device array of the library, GSW_STATIC_SCRATCH_BYTES (about
 * 24 MiB) per GPU that loads the library, held until the process exits.
 *
 * It computes what gsw_align_batch computes without GSW_BEGIN / GSW_CIGAR:
 * score1, ref_end1, read_end1, score2, ref_end2 (begins -1, no CIGAR), and
 * with GSW_COLMAX the per-column max array.  Arguments are as for
 * gsw_align_batch, device pointers only (no GSW_HOST_IO); flags may be 0 or
 * GSW_COLMAX.  max_target_len must be at least the longest t_len of the batch
 * and at most GSW_STATIC_MAX_TARGET (1024); larger values are rejected with
 * GSW_EINVAL before any work.  The kernel checks every pair before touching
 * its data, as gsw_align_batch does: a pair with a length outside [0, 2^24),
 * a negative offset (colmax_off too, with GSW_COLMAX), a target longer than
 * GSW_STATIC_MAX_TARGET or a letter code >= alphabet is not aligned; its
 * record is the empty one (score1 = 0, positions -1) flagged GSW_RES_INVALID,
 * and the call returns GSW_EINVAL after every other pair is done.
 *
 * The first call on a device looks up the device address of the array (and
 * sets the kernel's shared-memory limit); make that first call before any
 * stream capture.  Every call shares the one array and the call waits for its
 * stream before returning, so calls that overlap on the GPU (from several
 * host threads or streams at once) race and must be serialized by the caller.
 */
#define GSW_STATIC_MAX_TARGET 1024
#define GSW_STATIC_SCRATCH_BYTES (1216u * 1024u * 20u + 256u)
int gsw_fill_static(int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                    const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                    int32_t max_target_len, const int8_t *matrix, int32_t alphabet,
                    int32_t gap_open, int32_t gap_extend, uint32_t flags, int32_t mask_len,
                    gsw_result *results, int32_t *colmax, const int64_t *colmax_off,
                    void *stream);

/*
 * Serving loop (continuous batching).  A server owns `workers` batch slots,
 * each with its own context (scratch bounded by mem_budget_bytes / workers),
 * stream and pinned / device staging.  Requests (one or more pairs, host
 * memory, copied at submit) wait in a FIFO; a free worker forms its next
 * batch from the head of the queue -- as many whole requests as fit its
 * max_batch_pairs and max_batch_letters -- and runs the whole hot path on it
 * while the other workers' batches are on the GPU, so requests that arrive
 * while others are being aligned are admitted as soon as a slot frees.  Each
 * request's results are those gsw_align_batch gives for it alone.
 * Paper analogue: MOSAIK, SCISSORS and TANGRAM calling the library from many
 * threads at once (Applications).
 */
typedef struct gsw_server gsw_server;
typedef struct gsw_serve_config {
    int32_t device;
    int32_t workers;             /* batches in flight; 0 -> 4 */
    int32_t max_batch_pairs;     /* pairs per batch; 0 -> 8192 */
    int64_t max_batch_letters;   /* query + target letters per batch; 0 -> 16M */
    size_t mem_budget_bytes;     /* device memory of all workers; 0 -> 8 GiB */
    int32_t max_queue_requests;  /* queued requests beyond which submit fails (GSW_ENOMEM); 0 -> 1M */
    uint32_t flags;              /* GSW_BEGIN and/or GSW_CIGAR */
    int32_t mask_len;            /* as gsw_align_batch */
    const int8_t *matrix;        /* alphabet x alphabet, copied */
    int32_t alphabet, gap_open, gap_extend;
    /* Requests of at least heavy_cells cells (sum of m*n) queue apart and go
     * to the first heavy_workers workers, whose launches are sized for
     * heavy_sm_limit SMs; the other workers take only light requests, so a
     * short request never waits behind a long one.  heavy_workers 0 -> half
     * the workers (none if there is one), < 0 -> none; heavy_cells 0 -> 2^25,
     * heavy_sm_limit 0 -> 7/8 of the SMs, < 0 -> all. */
    int32_t heavy_workers;
    int64_t heavy_cells;
    int32_t heavy_sm_limit;
    /* When the light queue is keeping up (empty once a batch is formed), a
     * light worker pads a batch of at most 1024 pairs of at most 1024
     * letters a sequence to 64, 256 or 1024
     * pairs (with empty pairs) and rounds its largest lengths and traceback
     * scratch up to powers of four, so that batches of the same bucket
     * replay one captured CUDA graph of the pipeline instead of launching
     * each kernel; larger batches and batches formed under a backlog launch
     * eagerly.  0 -> on (default), < 0 -> off.  Results do not depend on it. */
    int32_t light_graphs;
} gsw_serve_config;

/* Starts the workers.  Errors: GSW_EINVAL (scoring, flags), GSW_ENOMEM, GSW_ECUDA. */
int gsw_serve_create(const gsw_serve_config *cfg, gsw_server **out);

/* Stops the workers after the queued and running batches finish. */
int gsw_serve_destroy(gsw_server *srv);

/* Queues one request of npairs pairs (layout of gsw_align_batch, host memory,
 * copied before return).  Errors: GSW_EINVAL (a request larger than one batch,
 * bad lengths or letters are reported by its poll), GSW_ENOMEM (queue full). */
int gsw_serve_submit(gsw_server *srv, int32_t npairs, const uint8_t *q, const int64_t *q_off,
                     const int32_t *q_len, const uint8_t *t, const int64_t *t_off,
                     const int32_t *t_len, uint64_t *req_id);

/* Waits at most timeout_us (< 0: no limit) for request req_id; on completion
 * copies its npairs records to `results` (host) and its CIGAR words to
 * `cigar` (cigar_off in the records index this buffer), sets *cigar_words,
 * and forgets the request.  Returns the request's status (GSW_OK or the error
 * of its batch), GSW_ETIMEDOUT (still queued or running; poll again),
 * GSW_ENOTFOUND, or GSW_ECIGAR_SPACE (cigar_capacity too small; the request
 * is kept).  Thread-safe with submit. */
int gsw_serve_poll(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_result *results,
                   uint32_t *cigar, int64_t cigar_capacity, int64_t *cigar_words);

/* gsw_serve_poll returning the request's records as a library-owned handle
 * (see gsw_align_batch_results; no max arrays); *out is set on GSW_OK and
 * GSW_EINTERNAL, and the request is forgotten.  Other returns as
 * gsw_serve_poll (GSW_ETIMEDOUT: poll again). */
int gsw_serve_poll_results(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_results **out);

/* Times of one request on the server's monotonic clock (seconds since
 * gsw_serve_create): queued by submit, taken into a batch by a worker, and
 * its batch's results on the host. */
typedef struct gsw_serve_times {
    double submitted, started, done;
} gsw_serve_times;

/* gsw_serve_poll that also fills *times (may be NULL) when the request is
 * complete. */
int gsw_serve_poll_timed(gsw_server *srv, uint64_t req_id, int32_t timeout_us, gsw_result *results,
                         uint32_t *cigar, int64_t cigar_capacity, int64_t *cigar_words,
                         gsw_serve_times *times);

/* The server's clock now (seconds since gsw_serve_create); -1 for NULL. */
double gsw_serve_now(gsw_server *srv);

typedef struct gsw_serve_stats {
    uint64_t submitted, completed, batches, pairs, cells;
    double busy_seconds;         /* sum over workers of time with a batch in flight */
    int32_t queued, running;
    uint64_t graph_batches;      /* batches whose pipeline replayed captured graphs */
} gsw_serve_stats;
int gsw_serve_get_stats(gsw_server *srv, gsw_serve_stats *out);

/* Name of an error code (static string). */
const char *gsw_strerror(int code);

/* Detail of the last error raised on the calling thread (static per thread). */
const char *gsw_last_error(void);

/* Library version string. */
const char *gsw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSW_H */
