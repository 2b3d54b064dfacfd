// Work planning for the persistent fill launches, entirely on the device so
// that a batch needs no host round trip and the stage chain can be captured
// in a CUDA graph.  A counting sort groups pairs by fill class (how many
// query rows a strip covers; queries of many strips go to the CTA kernel)
// and, inside a class, by estimated cost (strips x steps) descending; the
// persistent kernels then hand out tasks heaviest class first, so long pairs
// start early and the tail is made of short ones.
#include "gsw_impl.cuh"

#include <climits>

namespace gsw {
namespace {

constexpr int kScanThreads = 1024;


__device__ __forceinline__ int cost_bin(long long cost) {
    // 32 bins per doubling of cost, descending order inside a variant
    float lg = log2f((float)(cost < 1 ? 1 : cost));
    int bin = (int)(lg * 32.0f);
    bin = bin < 0 ? 0 : (bin > kPlanBinsPerVariant - 1 ? kPlanBinsPerVariant - 1 : bin);
    return kPlanBinsPerVariant - 1 - bin;
}

__global__ void k_plan_keys(BatchView b, Scoring sc, int32_t mode, int32_t *keys, int32_t *hist) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.npairs) return;
    int rows, cols, v;
    if (mode == kFillForward) {
        rows = b.q_len[p];
        cols = b.t_len[p];
        if (b.flags & GSW_FORCE_S32) v = (cols > 0 && long_pair(rows, true, sc.dna4)) ? kClassLong32 : kVarS32;
        else v = (cols > 0 && rows > 0) ? pick_class16(rows, sc) : 0;  // (any class writes an empty pair's record)
    } else if (mode == kFillRerun) {
        if (!(b.res[p].flags & kResPendingS32)) { keys[p] = -1; return; }
        rows = b.q_len[p];
        cols = b.t_len[p];
        v = long_pair(rows, true, sc.dna4) ? kClassLong32 : kVarS32;
    } else if (mode == kFillReverse) {
        // the ring fill takes the reverse of pairs whose band is too wide or
        // too long for one thread
        const gsw_result r = b.res[p];
        if (r.score1 <= 0 || (r.flags & kResInternal)) { keys[p] = -1; return; }
        rows = r.read_end1 + 1;
        const int wrev = reverse_band_width(r.read_end1, r.score1, sc);
        if (!small_batch(b) && wrev >= 0 && wrev <= kBandMaxRevWidth && rows <= kBandMaxRows) {
            keys[p] = -1;
            return;
        }
        cols = reverse_window(r.read_end1, r.ref_end1, r.score1, sc);
        // a query of several strips reverses in the CTA kernel: its strips run
        // concurrently, so the stop at the first column reaching score1 (often
        // a few dozen columns into a window of thousands) ends every strip,
        // where a group would finish the upper strips over the whole window
        // before the last one starts (4-letter DNA: a general alphabet's CTA
        // holds 4 warps per SM)
        v = pick_class_reverse(rows, (r.flags & GSW_RES_S32) != 0, sc);
    } else if (mode == kPlanTrace) {
        const gsw_result r = b.res[p];
        if (r.score1 <= 0 || !(r.flags & kResPendingTrace) || (r.flags & kResInternal) || r.read_begin1 < 0) {
            keys[p] = -1;
            return;
        }
        const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
        int dlo, dhi;
        // 0-3: anti-diagonal warp kernel (<= 64/128/256/512 diagonals); 4:
        // wider bands, the CTA strip kernel; 5-8: the 16-bit rectangle
        const int cls = trace_class(la, lb, r.score1, sc, small_batch(b), &dlo, &dhi);
        const int width = dhi - dlo + 1;
        const long long cost = cls >= kTraceT16First ? (long long)t16_strips(la, cls - kTraceT16First) * t16_steps(lb)
                                                     : (long long)(la + lb + 1) * ((width + 31) / 32);
        const int key = cls * kPlanBinsPerVariant + cost_bin(cost);
        keys[p] = key;
        atomicAdd(&hist[key], 1);
        return;
    } else {
        // kPlanBand: classes 0/1/2 = band width <= 8/16/32 diagonals
        const gsw_result r = b.res[p];
        if (r.score1 <= 0 || (r.flags & kResInternal)) { keys[p] = -1; return; }
        int width;
        if (r.read_begin1 < 0) {
            const int wrev = reverse_band_width(r.read_end1, r.score1, sc);
            rows = r.read_end1 + 1;
            width = wrev < 0 ? INT_MAX : wrev;
            if (width > kBandMaxRevWidth || rows > kBandMaxRows) {
                b.res[p].flags |= kResInternal;  // the ring reverse should have taken it
                keys[p] = -1;
                return;
            }
        } else {
            if (!(b.flags & GSW_CIGAR)) { keys[p] = -1; return; }
            const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
            int dlo, dhi;
            width = band_range(la, lb, r.score1, sc, &dlo, &dhi);
            rows = la;
            if (small_batch(b) || width > kBandMaxWidth || rows > kBandMaxRows) {
                b.res[p].flags |= kResPendingTrace;
                keys[p] = -1;
                return;
            }
        }
        const int cls = width <= 8 ? 0 : (width <= 16 ? 1 : 2);
        const int key = cls * kPlanBinsPerVariant + cost_bin(rows);
        keys[p] = key;
        atomicAdd(&hist[key], 1);
        return;
    }
    const Variant var = variant_at(v);
    const int sp = variant_rows(v);
    const long long strips = rows <= 0 ? 1 : (rows + sp - 1) / sp;
    const long long steps = (long long)cols + (var.s32 ? var.P : 2 * var.P);
    const int key = v * kPlanBinsPerVariant + cost_bin(strips * steps);
    keys[p] = key;
    atomicAdd(&hist[key], 1);
}

// Exclusive scan of the bins (one block), variant boundaries and task ranges.
__global__ void __launch_bounds__(kScanThreads) k_plan_scan(const int32_t *hist, int32_t *binoff,
                                                             int32_t *var_start, int32_t *task_lo,
                                                             int32_t *task_hi, int32_t *ntasks, int32_t *head) {
    constexpr int PER = kPlanBins / kScanThreads;
    static_assert(kPlanBins % kScanThreads == 0, "bins");
    __shared__ int32_t part[kScanThreads];
    const int tid = threadIdx.x;
    int32_t loc[PER];
    int32_t sum = 0;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        loc[i] = sum;
        sum += hist[tid * PER + i];
    }
    // inclusive scan of the threads' sums: within each warp by shuffles,
    // then over the warp totals by the first warp
    static_assert(kScanThreads == 32 * 32, "one warp scans the warp totals");
    __shared__ int32_t wsum[32];
    const int lane = tid & 31, warp = tid >> 5;
    int32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t v = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d) w += v;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    part[tid] = incl + (warp > 0 ? wsum[warp - 1] : 0);
    const int32_t base = part[tid] - sum;
#pragma unroll
    for (int i = 0; i < PER; i++) binoff[tid * PER + i] = base + loc[i];
    __syncthreads();
    if (tid == 0) {
        int32_t starts[kNumFillClasses + 1];
        for (int v = 0; v < kNumFillClasses; v++) starts[v] = binoff[v * kPlanBinsPerVariant];
        starts[kNumFillClasses] = part[kScanThreads - 1];
        for (int v = 0; v <= kNumFillClasses; v++) var_start[v] = starts[v];
        int32_t t = 0;
        for (int v = kNumFillClasses - 1; v >= 0; v--) {
            const int per = 32 / variant_at(v).P;
            const int32_t cnt = starts[v + 1] - starts[v];
            task_lo[v] = t;
            t += (cnt + per - 1) / per;
            task_hi[v] = t;
        }
        *ntasks = t;
        for (int v = 0; v < kNumFillClasses; v++) head[v] = 0;
    }
}

__global__ void k_plan_scatter(int32_t npairs, const int32_t *keys, const int32_t *binoff, int32_t *cursor,
                               int32_t *order) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int key = keys[p];
    if (key < 0) return;
    order[binoff[key] + atomicAdd(&cursor[key], 1)] = p;
}

}  // namespace

cudaError_t launch_plan(const BatchView &b, const Scoring &sc, int32_t mode, const PlanBuffers &pb,
                        cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(pb.hist, 0, sizeof(int32_t) * kPlanBins, st))) return e;
    if ((e = cudaMemsetAsync(pb.cursor, 0, sizeof(int32_t) * kPlanBins, st))) return e;
    const int nb = (b.npairs + 255) / 256;
    if (nb > 0) k_plan_keys<<<nb, 256, 0, st>>>(b, sc, mode, pb.keys, pb.hist);
    k_plan_scan<<<1, kScanThreads, 0, st>>>(pb.hist, pb.binoff, pb.var_start, pb.task_lo, pb.task_hi,
                                            pb.ntasks, pb.head);
    if (nb > 0) k_plan_scatter<<<nb, 256, 0, st>>>(b.npairs, pb.keys, pb.binoff, pb.cursor, pb.order);
    return cudaGetLastError();
}

}  // namespace gsw
