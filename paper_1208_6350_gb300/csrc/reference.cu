// Reads against one long reference (gsw_align_to_reference, include/gsw.h):
// the paper's alignments of reads to whole viral, bacterial and human
// chromosome sequences (Results, Performance), exact, on the batched path.
//
// Windows.  A local alignment of a read of m letters with a positive score
// covers at most m + D reference letters, D = (m*wmax - O)/X + 1 gap letters
// on the reference (each costs at least X after the first O).  The reference is
// cut into windows that own S consecutive columns and start V = m + D + 1
// columns earlier: every alignment ending in an owned column lies inside its
// window, so the window's DP values there are the full DP's; in the overlap
// they are lower bounds.  Merging the windows' (maximum, first column) pairs
// by larger score, then smaller column, therefore gives the full DP's score1
// and end column (the owner of the first column holding the maximum reports
// it exactly; any other report of that value is at a later column).  The
// secondary score is the same merge over the columns outside the mask around
// the end: windows whose range misses the mask contribute their (maximum,
// first column); the (at most three) whose range meets it are filled again
// with their max arrays and contribute the masked maximum.  A last pair, the
// read against the V columns ending at the end column, gives the end row (its
// DP is exact in its last column), the begin and the CIGAR.
//
// Passes: windows (score only) -> per-read merge -> windows at the mask
// (max arrays) -> masked merge -> end pairs (begin + CIGAR) -> results.
#include "gsw_impl.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace gsw {
namespace {

constexpr int kRefMaskSlots = 3;  // windows whose range can meet the mask

struct RefGeom {
    long long N;  // reference letters
    long long S;  // owned columns per window
    long long V;  // overlap
    int K;        // windows per read
    __host__ __device__ long long start(int k) const {
        const long long s = (long long)k * S - V;
        return s > 0 ? s : 0;
    }
    __host__ __device__ long long end(int k) const {
        const long long e = (long long)(k + 1) * S;
        return e < N ? e : N;
    }
};

__global__ void k_ref_windows(RefGeom g, int nreads, const int64_t *rq_off, const int32_t *rq_len, int64_t *qo,
                              int32_t *ql, int64_t *to, int32_t *tl) {
    const long long np = (long long)nreads * g.K;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(p / g.K), k = (int)(p % g.K);
        qo[p] = rq_off[r];
        ql[p] = rq_len[r];
        to[p] = g.start(k);
        tl[p] = (int32_t)(g.end(k) - g.start(k));
    }
}

__device__ __forceinline__ bool better(int v, long long c, int bv, long long bc) {
    return v > bv || (v == bv && v > 0 && c < bc);
}

// one warp per read: best (score, first global column) over its windows, and
// the same over the windows whose range misses the mask around that end
struct RefBest {
    int score1;
    long long end_t;
    int score_nt;      // best outside the mask, windows that miss it
    long long col_nt;
    long long mask_lo, mask_hi;  // masked reference columns (mask_lo > mask_hi: none)
    int kmask0;        // first window whose range meets the mask (-1: none)
};

__device__ __forceinline__ void warp_best(int &v, long long &c) {
    for (int d = 16; d; d >>= 1) {
        const int ov = __shfl_xor_sync(0xFFFFFFFFu, v, d);
        const long long oc = __shfl_xor_sync(0xFFFFFFFFu, c, d);
        if (better(ov, oc, v, c)) {
            v = ov;
            c = oc;
        }
    }
}

__global__ void k_ref_best(RefGeom g, int nreads, const int32_t *rq_len, int32_t mask_len, const gsw_result *wres,
                           RefBest *best) {
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nreads) return;
    const gsw_result *w = wres + (size_t)r * g.K;
    int v = 0;
    long long c = LLONG_MAX;
    for (int k = lane; k < g.K; k += 32) {
        const int s = w[k].score1;
        if (s > 0) {
            const long long col = g.start(k) + w[k].ref_end1;
            if (better(s, col, v, c)) {
                v = s;
                c = col;
            }
        }
    }
    warp_best(v, c);
    RefBest b;
    b.score1 = v;
    b.end_t = v > 0 ? c : -1;
    const int m = rq_len[r];
    const long long L = mask_len >= 0 ? mask_len : (m / 2 > 15 ? m / 2 : 15);
    if (v > 0) {
        b.mask_lo = c - L > 0 ? c - L : 0;
        b.mask_hi = c + L < g.N - 1 ? c + L : g.N - 1;
    } else {
        b.mask_lo = 1;
        b.mask_hi = 0;
    }
    // windows whose range [start, end) meets [mask_lo, mask_hi]
    int k0 = -1;
    if (b.mask_lo <= b.mask_hi) {
        k0 = (int)(b.mask_lo / g.S);
        while (k0 > 0 && g.end(k0 - 1) > b.mask_lo) k0--;
        while (k0 < g.K && g.end(k0) <= b.mask_lo) k0++;
    }
    b.kmask0 = k0;
    int v2 = 0;
    long long c2 = LLONG_MAX;
    for (int k = lane; k < g.K; k += 32) {
        const bool meets = b.mask_lo <= b.mask_hi && g.start(k) <= b.mask_hi && g.end(k) > b.mask_lo;
        const int s = w[k].score1;
        if (!meets && s > 0) {
            const long long col = g.start(k) + w[k].ref_end1;
            if (better(s, col, v2, c2)) {
                v2 = s;
                c2 = col;
            }
        }
    }
    warp_best(v2, c2);
    b.score_nt = v2;
    b.col_nt = c2;
    if (lane == 0) best[r] = b;
}

// pairs of the second pass: up to kRefMaskSlots windows per read that meet
// the mask (an empty target where there is none)
__global__ void k_ref_mask_pairs(RefGeom g, int nreads, const int64_t *rq_off, const int32_t *rq_len,
                                 const RefBest *best, int64_t *qo, int32_t *ql, int64_t *to, int32_t *tl,
                                 int64_t *cmoff, long long cm_stride) {
    const long long np = (long long)nreads * kRefMaskSlots;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(p / kRefMaskSlots), s = (int)(p % kRefMaskSlots);
        const RefBest b = best[r];
        const int k = b.kmask0 + s;
        const bool use = b.kmask0 >= 0 && k < g.K && g.start(k) <= b.mask_hi && g.end(k) > b.mask_lo;
        qo[p] = rq_off[r];
        ql[p] = rq_len[r];
        to[p] = use ? g.start(k) : 0;
        tl[p] = use ? (int32_t)(g.end(k) - g.start(k)) : 0;
        cmoff[p] = p * cm_stride;
    }
}

// masked maximum of the second pass's max arrays, merged with the windows
// that miss the mask: score2 and ref_end2
__global__ void k_ref_secondary(RefGeom g, int nreads, const RefBest *best, const int32_t *colmax, long long cm_stride,
                                int *sec, long long *sec_col) {
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nreads) return;
    const RefBest b = best[r];
    int v = b.score_nt;
    long long c = b.col_nt;
    if (b.kmask0 >= 0) {
        for (int s = 0; s < kRefMaskSlots; s++) {
            const int k = b.kmask0 + s;
            if (k >= g.K || g.start(k) > b.mask_hi || g.end(k) <= b.mask_lo) continue;
            const long long st = g.start(k), len = g.end(k) - st;
            const int32_t *cm = colmax + ((long long)r * kRefMaskSlots + s) * cm_stride;
            for (long long x = lane; x < len; x += 32) {
                const long long col = st + x;
                if (col >= b.mask_lo && col <= b.mask_hi) continue;
                const int val = cm[x];
                if (better(val, col, v, c)) {
                    v = val;
                    c = col;
                }
            }
        }
    }
    warp_best(v, c);
    if (lane == 0) {
        sec[r] = v;
        sec_col[r] = v > 0 ? c : -1;
    }
}

// the end pairs: the read against the V reference columns ending at its end
__global__ void k_ref_end_pairs(RefGeom g, int nreads, const int64_t *rq_off, const int32_t *rq_len,
                                const RefBest *best, int64_t *qo, int32_t *ql, int64_t *to, int32_t *tl) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreads; r += gridDim.x * blockDim.x) {
        const RefBest b = best[r];
        qo[r] = rq_off[r];
        ql[r] = b.score1 > 0 ? rq_len[r] : 0;
        const long long s = b.score1 > 0 && b.end_t > g.V ? b.end_t - g.V : 0;
        to[r] = s;
        tl[r] = b.score1 > 0 ? (int32_t)(b.end_t - s + 1) : 0;
    }
}

__global__ void k_ref_finish(int nreads, const RefBest *best, const int *sec, const long long *sec_col,
                             const int64_t *end_to, gsw_result *res) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreads; r += gridDim.x * blockDim.x) {
        const RefBest b = best[r];
        gsw_result x = res[r];  // the end pair's record (begin, CIGAR, end row)
        if (b.score1 <= 0) {
            x.score1 = 0;
            x.ref_begin1 = x.ref_end1 = x.read_begin1 = x.read_end1 = -1;
            x.cigar_len = 0;
            x.cigar_off = -1;
        } else {
            // the end pair's own end must be its last column, with score1
            if (x.score1 != b.score1 || end_to[r] + x.ref_end1 != b.end_t) x.flags |= kResInternal;
            x.ref_end1 = (int32_t)b.end_t;
            if (x.ref_begin1 >= 0) x.ref_begin1 = (int32_t)(end_to[r] + x.ref_begin1);
        }
        x.score2 = sec[r];
        x.ref_end2 = (int32_t)sec_col[r];
        res[r] = x;
    }
}

int grid_for(long long n) { return (int)std::max(1LL, std::min(8192LL, (n + 255) / 256)); }

}  // namespace
}  // namespace gsw

extern "C" int gsw_align_to_reference(gsw_ctx *ctx, int32_t nreads, const uint8_t *q, const int64_t *q_off,
                                      const int32_t *q_len, const uint8_t *ref, int64_t ref_len,
                                      const int8_t *matrix, int32_t alphabet, int32_t gap_open, int32_t gap_extend,
                                      uint32_t flags, int32_t mask_len, int64_t window, gsw_result *results,
                                      uint32_t *cigar, int64_t cigar_capacity, void *stream) {
    using namespace gsw;
    if (!ctx || nreads < 0 || ref_len < 0 || ref_len >= (1LL << 31) || !matrix || window < 0)
        return set_err(GSW_EINVAL, "context, read count, reference length (< 2^31), matrix or window");
    if (flags & ~(GSW_BEGIN | GSW_CIGAR | GSW_HOST_IO)) return set_err(GSW_EINVAL, "unknown flag bits 0x%x", flags);
    if (nreads == 0) return GSW_OK;
    if (!q || !q_off || !q_len || !results || (ref_len > 0 && !ref)) return set_err(GSW_EINVAL, "NULL input or result pointer");
    if ((flags & GSW_CIGAR) && !cigar && cigar_capacity > 0) return set_err(GSW_EINVAL, "cigar is NULL");
    {
        Scoring chk;
        const int e = make_scoring(matrix, alphabet, gap_open, gap_extend, &chk);
        if (e != GSW_OK) return e;
    }
    int wmax = -128;
    for (int i = 0; i < alphabet * alphabet; i++) wmax = std::max<int>(wmax, matrix[i]);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(context_device(ctx)) != cudaSuccess) return set_err(GSW_ECUDA, "cudaSetDevice");
    const bool hio = (flags & GSW_HOST_IO) != 0;
    // read lengths on the host (the window geometry depends on the longest)
    std::vector<int32_t> hql(nreads);
    std::vector<int64_t> hqo(nreads);
    if (hio) {
        std::copy(q_len, q_len + nreads, hql.begin());
        std::copy(q_off, q_off + nreads, hqo.begin());
    } else if (cudaMemcpyAsync(hql.data(), q_len, 4 * (size_t)nreads, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess) {
        // read on the call's stream: work queued there before the call may write the lengths
        return set_err(GSW_ECUDA, "read-length readback");
    }
    int maxm = 0;
    int64_t qext = 0;
    for (int r = 0; r < nreads; r++) {
        if (hql[r] < 0 || hql[r] >= (1 << 24)) return set_err(GSW_EINVAL, "read %d: length out of [0, 2^24)", r);
        maxm = std::max(maxm, hql[r]);
        if (hio) qext = std::max<int64_t>(qext, hqo[r] + hql[r]);
    }
    RefGeom g;
    g.N = ref_len;
    long long D = gap_extend > 0 ? ((long long)maxm * std::max(wmax, 0) - gap_open) / gap_extend + 1 : ref_len;
    g.V = std::min<long long>(ref_len, (long long)maxm + std::max(0LL, D) + 1);
    // the mask around an end meets at most 2 windows when S > 2L + V
    const long long Lmax = mask_len >= 0 ? mask_len : std::max(maxm / 2, 15);
    const long long Smin = 2 * Lmax + g.V + 1;
    if (window > 0 && window < Smin) return set_err(GSW_EINVAL, "window %lld < 2 x mask + overlap + 1 = %lld", (long long)window, Smin);
    g.S = window > 0 ? window : std::max({65536LL, 4 * g.V, Smin});
    g.K = (int)std::max(1LL, (ref_len + g.S - 1) / g.S);
    if ((long long)nreads * g.K >= (1LL << 31) || g.S + g.V >= (1LL << 24))
        return set_err(GSW_EINVAL, "reads x windows >= 2^31 or window + overlap >= 2^24");
    const long long np = (long long)nreads * g.K;

    // device buffers (plain allocations for this call)
    uint8_t *dq = nullptr, *dref = nullptr;
    int64_t *drqo = nullptr, *wqo = nullptr, *wto = nullptr, *cmoff = nullptr, *eqo = nullptr, *eto = nullptr;
    int32_t *drql = nullptr, *wql = nullptr, *wtl = nullptr, *colmax = nullptr, *eql = nullptr, *etl = nullptr;
    gsw_result *wres = nullptr, *mres = nullptr, *eres = nullptr;
    RefBest *best = nullptr;
    int *sec = nullptr;
    long long *sec_col = nullptr;
    uint32_t *dcig = nullptr;
    unsigned long long *nflag = nullptr, hflag = 0;
    const long long cm_stride = (g.S + g.V + 3) / 4 * 4;
    const long long nm = (long long)nreads * kRefMaskSlots;
    int rc = GSW_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (rc == GSW_OK && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = GSW_ENOMEM;
    };
    if (hio) {
        alloc((void **)&dq, (size_t)std::max<int64_t>(qext, 1));
        alloc((void **)&dref, (size_t)std::max<int64_t>(ref_len, 1));
        alloc((void **)&drqo, 8 * (size_t)nreads);
        alloc((void **)&drql, 4 * (size_t)nreads);
        if (flags & GSW_CIGAR) alloc((void **)&dcig, 4 * (size_t)std::max<int64_t>(cigar_capacity, 1));
    }
    // the window pair arrays serve pass 1 (np pairs) and pass 2 (nm pairs)
    const long long npm = std::max(np, nm);
    alloc((void **)&wqo, 8 * (size_t)npm);
    alloc((void **)&wto, 8 * (size_t)npm);
    alloc((void **)&wql, 4 * (size_t)npm);
    alloc((void **)&wtl, 4 * (size_t)npm);
    alloc((void **)&wres, sizeof(gsw_result) * (size_t)np);
    alloc((void **)&best, sizeof(RefBest) * (size_t)nreads);
    alloc((void **)&cmoff, 8 * (size_t)nm);
    alloc((void **)&colmax, 4 * (size_t)(nm * cm_stride));
    alloc((void **)&mres, sizeof(gsw_result) * (size_t)nm);
    alloc((void **)&sec, sizeof(int) * (size_t)nreads);
    alloc((void **)&sec_col, sizeof(long long) * (size_t)nreads);
    alloc((void **)&eqo, 8 * (size_t)nreads);
    alloc((void **)&eto, 8 * (size_t)nreads);
    alloc((void **)&eql, 4 * (size_t)nreads);
    alloc((void **)&etl, 4 * (size_t)nreads);
    alloc((void **)&eres, sizeof(gsw_result) * (size_t)nreads);
    alloc((void **)&nflag, sizeof(unsigned long long));
    const uint8_t *Q = q, *R = ref;
    const int64_t *RQO = q_off;
    const int32_t *RQL = q_len;
    gsw_result *RES = hio ? eres : results;
    uint32_t *CIG = hio ? dcig : cigar;
    if (rc == GSW_OK && hio) {
        bool ok = cudaMemcpyAsync(dq, q, (size_t)qext, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                  cudaMemcpyAsync(dref, ref, (size_t)ref_len, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                  cudaMemcpyAsync(drqo, q_off, 8 * (size_t)nreads, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                  cudaMemcpyAsync(drql, q_len, 4 * (size_t)nreads, cudaMemcpyHostToDevice, st) == cudaSuccess;
        if (!ok) rc = GSW_ECUDA;
        Q = dq;
        R = dref;
        RQO = drqo;
        RQL = drql;
    }
    // pass 1: every window, score only
    if (rc == GSW_OK) {
        k_ref_windows<<<grid_for(np), 256, 0, st>>>(g, nreads, RQO, RQL, wqo, wql, wto, wtl);
        rc = gsw_align_batch(ctx, (int32_t)np, Q, wqo, wql, R, wto, wtl, matrix, alphabet, gap_open, gap_extend, 0,
                             mask_len, wres, nullptr, 0, nullptr, nullptr, stream);
    }
    // merge per read; pass 2: the windows at the mask, with their max arrays
    if (rc == GSW_OK) {
        k_ref_best<<<(nreads * 32 + 255) / 256, 256, 0, st>>>(g, nreads, RQL, mask_len, wres, best);
        k_ref_mask_pairs<<<grid_for(nm), 256, 0, st>>>(g, nreads, RQO, RQL, best, wqo, wql, wto, wtl, cmoff,
                                                       cm_stride);
        rc = gsw_align_batch(ctx, (int32_t)nm, Q, wqo, wql, R, wto, wtl, matrix, alphabet, gap_open, gap_extend,
                             GSW_COLMAX, mask_len, mres, nullptr, 0, colmax, cmoff, stream);
    }
    if (rc == GSW_OK) {
        k_ref_secondary<<<(nreads * 32 + 255) / 256, 256, 0, st>>>(g, nreads, best, colmax, cm_stride, sec, sec_col);
        // pass 3: the end pairs give the end row, the begin and the CIGAR
        k_ref_end_pairs<<<grid_for(nreads), 256, 0, st>>>(g, nreads, RQO, RQL, best, eqo, eql, eto, etl);
        const uint32_t f3 = flags & (GSW_BEGIN | GSW_CIGAR);
        rc = gsw_align_batch(ctx, nreads, Q, eqo, eql, R, eto, etl, matrix, alphabet, gap_open, gap_extend, f3,
                             mask_len, RES, (f3 & GSW_CIGAR) ? CIG : nullptr, (f3 & GSW_CIGAR) ? cigar_capacity : 0,
                             nullptr, nullptr, stream);
    }
    int rc_cigar = GSW_OK;
    if (rc == GSW_ECIGAR_SPACE || rc == GSW_EINTERNAL) {
        // records are complete; the caller learns the space needed (the
        // internal flags are counted again below, after the merge)
        if (rc == GSW_ECIGAR_SPACE) rc_cigar = rc;
        rc = GSW_OK;
    }
    if (rc == GSW_OK) {
        k_ref_finish<<<grid_for(nreads), 256, 0, st>>>(nreads, best, sec, sec_col, eto, RES);
        if (cudaMemsetAsync(nflag, 0, sizeof(unsigned long long), st) != cudaSuccess ||
            launch_count_flag(RES, nreads, kResInternal, nflag, st) != cudaSuccess ||
            cudaMemcpyAsync(&hflag, nflag, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = GSW_ECUDA;
    }
    if (rc == GSW_OK && hio) {
        bool ok = cudaMemcpyAsync(results, eres, sizeof(gsw_result) * (size_t)nreads, cudaMemcpyDeviceToHost, st) ==
                  cudaSuccess;
        if (ok && (flags & GSW_CIGAR) && cigar_capacity > 0)
            ok = cudaMemcpyAsync(cigar, dcig, 4 * (size_t)cigar_capacity, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (!ok) rc = GSW_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == GSW_OK) rc = GSW_ECUDA;
    void *bufs[] = {dq, dref, drqo, drql, dcig, wqo, wto, wql, wtl, wres, best, cmoff, colmax, mres,
                    sec, sec_col, eqo, eto, eql, etl, eres, nflag};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (rc == GSW_OK && hflag)
        return set_err(GSW_EINTERNAL, "%llu reads failed a consistency check (GSW_RES_INTERNAL)", hflag);
    return rc != GSW_OK ? rc : rc_cigar;
}
