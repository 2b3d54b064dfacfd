// Banded global Gotoh between begin and end, with the traceback that emits the
// CIGAR on the device ("Algorithm and implementation", item (1): the detailed
// alignment comes from a banded SW whose band the begin and the end fix), for
// bands of at most 512 diagonals (wider bands:
// trace_ring.cu; at most 32 diagonals and 4096 rows: band.cu).
//
// The band is the provable one (band_range): every diagonal that can carry a
// path scoring score1.  Inside it, every cell of every optimal path has the
// value of the full-rectangle DP, so each traceback comparison decides exactly
// as on the full rectangle and the CIGAR is the canonical one.
//
// One warp per pair, anti-diagonal by anti-diagonal: lane l holds diagonals
// 2l and 2l+1 of each chunk of 64 (NCH chunks, in registers), so a cell's
// left and upper neighbours are the adjacent diagonals of the previous
// anti-diagonal (one lane rotation), its diagonal neighbour the same diagonal
// two anti-diagonals back.  Each cell's 4 decision bits (H source diagonal /
// E / F; E opened here; F opened here) go to a per-lane word holding 8
// anti-diagonals, written every 8th anti-diagonal (128 contiguous bytes per
// chunk); the walk back from (la, lb) stages them through shared memory.  The
// pair's letters are staged in shared memory when they fit.
#include "gsw_impl.cuh"

#include <climits>

namespace gsw {
namespace {

constexpr int kTBlock = 128;
constexpr int kNegT = -(1 << 28);
constexpr int kNegHalf = -(1 << 27);
constexpr int kAdLetters = 2048;  // per warp: query + target letters staged in shared memory

// decision words of one pair: 8 anti-diagonals per word row, NCH x 32 words a row
__host__ __device__ inline long long ad_dir_words(int la, int lb, int nch) {
    return ((long long)(la + lb + 1 + 7) / 8) * nch * 32;
}

// pairs the thread-per-pair band kernel left to the warp tracebacks (band wider than 32)
__device__ __forceinline__ bool wants_trace(const gsw_result &r) {
    return r.score1 > 0 && (r.flags & kResPendingTrace) && !(r.flags & kResInternal) && r.read_begin1 >= 0 &&
           r.ref_begin1 >= 0;
}

// Largest needs of a pair of the warp classes: [0] direction words of the
// anti-diagonal classes, [1] op words (anti-diagonal and 16-bit classes);
// need16[v]: direction words of 16-bit class v (per group of 8 lanes).
__global__ void k_trace_need(BatchView b, Scoring sc, unsigned long long *max_need, unsigned long long *need16) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v[2 + kTraceT16Classes] = {};
    if (p < b.npairs) {
        const gsw_result r = b.res[p];
        if (wants_trace(r)) {
            const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
            int dlo, dhi;
            const int cls = trace_class(la, lb, r.score1, sc, small_batch(b), &dlo, &dhi);
            if (cls < kTraceRingClass) {
                v[0] = (unsigned)min(ad_dir_words(la, lb, 1 << cls), (long long)UINT_MAX);
                v[1] = (unsigned)min((long long)la + lb + 2, (long long)UINT_MAX);
            } else if (cls >= kTraceT16First) {
                v[2 + cls - kTraceT16First] =
                    (unsigned)min(t16_need_words(la, lb, cls - kTraceT16First), (long long)UINT_MAX);
                v[1] = (unsigned)min((long long)la + lb + 2, (long long)UINT_MAX);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 2 + kTraceT16Classes; k++) {
        const unsigned m = __reduce_max_sync(0xFFFFFFFFu, v[k]);
        if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(k < 2 ? &max_need[k] : &need16[k - 2], (unsigned long long)m);
    }
}

template <int NCH>
__device__ void trace_ad_pair(const BatchView &b, const Scoring &sc, const int8_t *sW, int p, const gsw_result &r,
                              int dlo, int dhi, uint32_t *dirs, uint32_t *ops, uint32_t *stage, uint8_t *lsm,
                              int lane) {
    const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
    const uint8_t *qs = b.q + b.q_off[p] + r.read_begin1;
    const uint8_t *ts = b.t + b.t_off[p] + r.ref_begin1;
    const int O = sc.O, X = sc.X, A = sc.A;
    // the pair's letters (clamped to the alphabet) in shared memory when they
    // fit: every cell reads two
    const bool staged = la + lb <= kAdLetters;
    if (staged) {
        for (int x = lane; x < la; x += 32) lsm[x] = (uint8_t)min((int)qs[x], A - 1);
        for (int x = lane; x < lb; x += 32) lsm[la + x] = (uint8_t)min((int)ts[x], A - 1);
        __syncwarp();
    }
    int H1[NCH], E1[NCH], F1[NCH], H2[NCH];
    uint32_t bits[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) { H1[c] = kNegT; E1[c] = kNegT; F1[c] = kNegT; H2[c] = kNegT; bits[c] = 0; }
    int final_h = kNegT;
    const int steps = la + lb;
    for (int a = 0; a <= steps; a++) {
        const int par = (a - dlo) & 1;
        // neighbour values from the previous anti-diagonal (before any
        // update): one lane rotation per value; the end lane sends its
        // neighbour chunk's value where the other end lane needs it
        int nh[NCH], nx[NCH];  // par 0: left (H, E); par 1: up (H, F)
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            if (par == 0) {
                const int sh = lane == 31 ? (c > 0 ? H1[c > 0 ? c - 1 : 0] : kNegT) : H1[c];
                const int se = lane == 31 ? (c > 0 ? E1[c > 0 ? c - 1 : 0] : kNegT) : E1[c];
                nh[c] = __shfl_sync(0xFFFFFFFFu, sh, (lane + 31) & 31);
                nx[c] = __shfl_sync(0xFFFFFFFFu, se, (lane + 31) & 31);
            } else {
                const int sh = lane == 0 ? (c + 1 < NCH ? H1[c + 1 < NCH ? c + 1 : c] : kNegT) : H1[c];
                const int sf = lane == 0 ? (c + 1 < NCH ? F1[c + 1 < NCH ? c + 1 : c] : kNegT) : F1[c];
                nh[c] = __shfl_sync(0xFFFFFFFFu, sh, (lane + 1) & 31);
                nx[c] = __shfl_sync(0xFFFFFFFFu, sf, (lane + 1) & 31);
            }
        }
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            const int d = dlo + 64 * c + 2 * lane + par;
            const int i = (a - d) >> 1, j = (a + d) >> 1;
            const bool valid = d <= dhi && (unsigned)i <= (unsigned)la && (unsigned)j <= (unsigned)lb;
            int hl, el, hu, fu;
            if (par == 0) { hl = nh[c]; el = nx[c]; hu = H1[c]; fu = F1[c]; }
            else { hl = H1[c]; el = E1[c]; hu = nh[c]; fu = nx[c]; }
            const int eo = hl - O, fo = hu - O;
            int E = j >= 1 ? max(eo, el - X) : kNegT;
            int F = i >= 1 ? max(fo, fu - X) : kNegT;
            const bool eopen = j >= 1 && E == eo, fopen = i >= 1 && F == fo;
            int hdg = kNegT;
            if (valid && i >= 1 && j >= 1) {
                const int qa = staged ? (int)lsm[i - 1] : min((int)qs[i - 1], A - 1);
                const int tb = staged ? (int)lsm[la + j - 1] : min((int)ts[j - 1], A - 1);
                hdg = H2[c] + sW[qa * A + tb];
            }
            int H = max(hdg, max(E, F));
            if (i == 0 && j == 0) H = 0;
            if (!valid || H < kNegHalf) { H = kNegT; E = kNegT; F = kNegT; }
            const uint32_t src = (hdg > kNegHalf && H == hdg) ? 0u : (H == E ? 1u : 2u);
            // 4 decision bits per cell; lane l of chunk c keeps 8 anti-diagonals
            // in one word (nibble a & 7), written every 8th one
            bits[c] |= (src | (eopen ? 4u : 0u) | (fopen ? 8u : 0u)) << (4 * (a & 7));
            if (valid && i == la && j == lb) final_h = H;
            H2[c] = H1[c];
            H1[c] = H;
            E1[c] = E;
            F1[c] = F;
        }
        if ((a & 7) == 7 || a == steps) {
#pragma unroll
            for (int c = 0; c < NCH; c++) {
                dirs[((size_t)(a >> 3) * NCH + c) * 32 + lane] = bits[c];
                bits[c] = 0;
            }
        }
    }
    final_h = __reduce_max_sync(0xFFFFFFFFu, final_h);
    __syncwarp();
    gsw_result *rp = b.res + p;
    // Walk back from (la, lb).  The anti-diagonal index i + j never increases
    // along the walk, so the warp stages the decision words into shared
    // memory 4 word rows (32 anti-diagonals) at a time, coalesced, and lane 0
    // walks inside the staged block; the runs go to `ops` in reverse order.
    constexpr int KROWS = 4;
    int i = la, j = lb, state = 0, cur = -1, len = 0, runs = 0;
    bool ok = final_h == r.score1;
    int row_hi = (la + lb) >> 3;
    while (ok && (i > 0 || j > 0) && row_hi >= 0) {
        const int row_lo = max(0, row_hi - KROWS + 1);
        const int nwords = (row_hi - row_lo + 1) * NCH * 32;
        for (int w = lane; w < nwords; w += 32) stage[w] = dirs[(size_t)row_lo * NCH * 32 + w];
        __syncwarp();
        if (lane == 0) {
            while ((i > 0 || j > 0) && ((i + j) >> 3) >= row_lo) {
                const int off2 = j - i - dlo;
                if (i < 0 || j < 0 || off2 < 0 || off2 >= 64 * NCH) { ok = false; break; }
                const int ad = i + j;
                const uint32_t wd =
                    stage[(((ad >> 3) - row_lo) * NCH + (off2 >> 6)) * 32 + ((off2 & 63) >> 1)] >> (4 * (ad & 7));
                const int src = wd & 3, eo = (wd >> 2) & 1, fo = (wd >> 3) & 1;
                int op;
                if (state == 0) {
                    if (src == 0) { op = GSW_CIGAR_M; i--; j--; }
                    else { state = src; continue; }
                } else if (state == 1) {
                    op = GSW_CIGAR_D; state = eo ? 0 : 1; j--;
                } else {
                    op = GSW_CIGAR_I; state = fo ? 0 : 2; i--;
                }
                if (op == cur) {
                    len++;
                } else {
                    if (len) ops[runs++] = ((uint32_t)len << 4) | (uint32_t)cur;
                    cur = op;
                    len = 1;
                }
            }
        }
        ok = __shfl_sync(0xFFFFFFFFu, (int)ok, 0);
        i = __shfl_sync(0xFFFFFFFFu, i, 0);
        j = __shfl_sync(0xFFFFFFFFu, j, 0);
        __syncwarp();
        row_hi = row_lo - 1;
    }
    if (lane == 0 && ok && (i != 0 || j != 0)) ok = false;
    if (lane == 0 && ok && len) ops[runs++] = ((uint32_t)len << 4) | (uint32_t)cur;
    ok = __shfl_sync(0xFFFFFFFFu, (int)ok, 0);
    const int nr = __shfl_sync(0xFFFFFFFFu, runs, 0);
    if (!ok) {
        if (lane == 0) rp->flags |= kResInternal;
        __syncwarp();
        return;
    }
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(b.cigar_cursor, (unsigned long long)nr);
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    if ((long long)(off + nr) > b.cigar_cap) {
        if (lane == 0) {
            rp->flags |= GSW_RES_CIGAR_SPACE;
            rp->cigar_len = -nr;
            rp->cigar_off = -1;
            rp->flags &= ~kResPendingTrace;
        }
        __syncwarp();
        return;
    }
    __syncwarp();
    for (int t = lane; t < nr; t += 32) b.cigar[off + t] = ops[nr - 1 - t];
    if (lane == 0) {
        rp->cigar_len = nr;
        rp->cigar_off = (int64_t)off;
        rp->flags &= ~kResPendingTrace;
    }
    __syncwarp();
}

template <int NCH>
__global__ void __launch_bounds__(kTBlock) k_trace_ad(BatchView b, Scoring sc, TraceScratch ts, int cls) {
    __shared__ int8_t sW[kMaxAlpha * kMaxAlpha];
    __shared__ uint32_t stage_all[kTBlock / 32][4 * NCH * 32];
    __shared__ uint8_t letters_all[kTBlock / 32][kAdLetters];
    for (int i = threadIdx.x; i < sc.A * sc.A; i += blockDim.x) sW[i] = sc.W[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (kTBlock / 32) + warp;
    const int nwarps = gridDim.x * (kTBlock / 32);
    uint32_t *dirs = ts.dirs + (size_t)gwarp * ts.dir_words;
    uint32_t *ops = ts.ops + (size_t)gwarp * ts.op_words;
    const int first = ts.var_start[cls], last = ts.var_start[cls + 1];
    for (int idx = first + gwarp; idx < last; idx += nwarps) {
        const int p = ts.order[idx];
        const gsw_result r = b.res[p];
        if (!wants_trace(r)) continue;
        const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
        int dlo, dhi;
        band_range(la, lb, r.score1, sc, &dlo, &dhi);
        if (ad_dir_words(la, lb, NCH) > ts.dir_words || dhi - dlo + 1 > 64 * NCH ||
            (long long)(la + lb + 2) > ts.op_words) {
            if (lane == 0) b.res[p].flags |= kResInternal;
            continue;
        }
        trace_ad_pair<NCH>(b, sc, sW, p, r, dlo, dhi, dirs, ops, stage_all[warp], letters_all[warp], lane);
        __syncwarp();
    }
}

}  // namespace


cudaError_t launch_trace_ad(const BatchView &b, const Scoring &sc, const TraceScratch &ts, int grid,
                            cudaStream_t st) {
    k_trace_ad<1><<<grid, kTBlock, 0, st>>>(b, sc, ts, 0);
    k_trace_ad<2><<<grid, kTBlock, 0, st>>>(b, sc, ts, 1);
    k_trace_ad<4><<<grid, kTBlock, 0, st>>>(b, sc, ts, 2);
    k_trace_ad<8><<<grid, kTBlock, 0, st>>>(b, sc, ts, 3);
    return cudaGetLastError();
}

int trace_block_threads() { return kTBlock; }

// Largest needs of the anti-diagonal classes: [0] direction words, [1] op words.
cudaError_t launch_trace_need(const BatchView &b, const Scoring &sc, unsigned long long *max_need,
                              unsigned long long *need16, cudaStream_t st) {
    cudaMemsetAsync(max_need, 0, 2 * sizeof(unsigned long long), st);
    cudaMemsetAsync(need16, 0, kTraceT16Classes * sizeof(unsigned long long), st);
    const int nb = (b.npairs + 255) / 256;
    if (nb > 0) k_trace_need<<<nb, 256, 0, st>>>(b, sc, max_need, need16);
    return cudaGetLastError();
}

}  // namespace gsw
