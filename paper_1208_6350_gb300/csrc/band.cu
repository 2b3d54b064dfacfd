// Begin and CIGAR for pairs whose bands are narrow: one thread per pair.
//
// Reversed SW from the end ("Algorithm and implementation", item (1)), as a
// banded DP.  Every alignment scoring score1 inside the rectangle
// q[0..end_q] x t[0..end_t] ends exactly at (end_q, end_t) (the end is the
// first column, then first row, holding score1).  On the reversed sequences
// these alignments all start at the origin, so the cells that reach score1 are
// the same in the local DP and in the DP anchored at the origin (no restarts),
// and an anchored path reaching score1 has at most
// G = ((end_q+1)*wmax - score1 - O)/X + 1 gap letters, hence never leaves the
// diagonals |j - i| <= G.  The anchored banded DP therefore finds the same
// first column (then first row) holding score1 as the full local reversed DP.
//
// Banded SW between begin and end (item (1)): global Gotoh restricted to the
// provable band (band_halfwidth), with 4 decision bits per cell and the same
// traceback preferences as the oracle.  The bits of a cell: H differs from the
// diagonal term (bit 0), H differs from E (bit 1), E extends rather than opens
// (bit 2), F extends rather than opens (bit 3).  The DP keeps H as H - O, so
// the opening candidates of E and F are stored values.  The traceback band is never wider than
// the reverse band (it bounds the same gap letters with fewer aligned pairs).
//
// Lanes of a warp take consecutive pairs of a list sorted by rows, so their
// loops have similar lengths.  Each lane keeps its band row in registers
// (W cells) and stores each row's decision nibbles into a per-warp scratch
// interleaved by lane (coalesced).  The walk keeps the first 16 runs it finds
// (the CIGAR's last ones) and counts the rest; a CIGAR of at most 16 runs is
// then written from them in forward order at the reserved offset, a longer
// one is walked a second time into its reserved words.
#include "gsw_impl.cuh"

#include <algorithm>

namespace gsw {
namespace {

constexpr int kBBlock = 128;
constexpr int kNegB = -(1 << 28);
constexpr int kNegBHalf = -(1 << 27);

template <int W>
struct DirWord;
template <>
struct DirWord<8> {
    using T = uint32_t;
};
template <>
struct DirWord<16> {
    using T = uint2;
};
template <>
struct DirWord<32> {
    using T = uint4;
};

template <int W>
__device__ __forceinline__ void put_nib(typename DirWord<W>::T &w, int k, uint32_t nib) {
    if constexpr (W == 8) {
        w |= nib << (4 * k);
    } else if constexpr (W == 16) {
        if (k < 8) w.x |= nib << (4 * k);
        else w.y |= nib << (4 * (k - 8));
    } else {
        const int s = 4 * (k & 7);
        if (k < 8) w.x |= nib << s;
        else if (k < 16) w.y |= nib << s;
        else if (k < 24) w.z |= nib << s;
        else w.w |= nib << s;
    }
}

// The 32-bit word of w that holds nibble k.
template <int W>
__device__ __forceinline__ uint32_t &nib_word(typename DirWord<W>::T &w, int k) {
    if constexpr (W == 8) return w;
    else if constexpr (W == 16) return k < 8 ? w.x : w.y;
    else return k < 8 ? w.x : k < 16 ? w.y : k < 24 ? w.z : w.w;
}

// bits |= m when a != b: a compare into a predicate and a predicated or
__device__ __forceinline__ void or_if_ne(uint32_t &bits, int a, int b, uint32_t m) {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(bits)
        : "r"(a), "r"(b), "r"(m));
}

template <int W>
__device__ __forceinline__ uint32_t get_nib(const typename DirWord<W>::T &w, int k) {
    if constexpr (W == 8) {
        return (w >> (4 * k)) & 15u;
    } else if constexpr (W == 16) {
        return ((k < 8 ? w.x : w.y) >> (4 * (k & 7))) & 15u;
    } else {
        const uint32_t v = k < 8 ? w.x : k < 16 ? w.y : k < 24 ? w.z : w.w;
        return (v >> (4 * (k & 7))) & 15u;
    }
}

template <int W>
__device__ __forceinline__ void zero(typename DirWord<W>::T &w) {
    if constexpr (W == 8) w = 0u;
    else if constexpr (W == 16) w = make_uint2(0u, 0u);
    else w = make_uint4(0u, 0u, 0u, 0u);
}

struct BandSeq {
    const uint8_t *q;  // row i (1-based) letter at q[(i-1) * qs]
    int qs;
    int rows;
    const uint8_t *t;  // column j (1-based) letter at t[(j-1) * ts]
    int ts;
    int cols;
};

// Banded global-start DP over rows 0..rows, band diagonals [dlo, dlo + wb).
// REV: finds the first column (then row) holding `target`; returns false if
// none.  !REV: stores decision nibbles per row and returns H(rows, cols).
template <int W, bool REV, bool DNA>
__device__ bool band_dp(const BandSeq &s, int dlo, int wb, const int8_t *sW, int A, int O, int X, int target,
                        typename DirWord<W>::T *dirs, int *out_i, int *out_j, int *final_h, int rstride = 32) {
    int Hp[W], Fp[W];  // H - O and F of the previous row's band cells
    int tw[W];  // target letter (DNA: 8 x letter, a byte shift) of each band cell's column in the current row
    constexpr int TM = DNA ? 8 : 1;
    const int negho = kNegB - O;  // H - O of a cell outside
#pragma unroll
    for (int k = 0; k < W; k++) {
        Hp[k] = negho;
        Fp[k] = kNegB;
        const int jj = dlo + k - 1;  // row 0: letter index j - 1 = dlo + k - 1 (shifted in before use)
        tw[k] = (jj >= 0 && jj < s.cols) ? TM * min((int)s.t[(long long)jj * s.ts], A - 1) : 0;
    }
    int best_j = INT_MAX, best_i = -1;
    int fin = kNegB;
    // the letters of row i+1 are loaded during row i
    auto qletter = [&](int i) { return i >= 1 && i <= s.rows ? min((int)s.q[(long long)(i - 1) * s.qs], A - 1) : 0; };
    auto tletter = [&](int i) {
        const int jj = i + dlo + W - 2;
        return (jj >= 0 && jj < s.cols) ? TM * min((int)s.t[(long long)jj * s.ts], A - 1) : 0;
    };
    int qa_next = qletter(1), tn_next = tletter(1);
    typename DirWord<W>::T *drow = dirs;
    for (int i = 0; i <= s.rows; i++) {
        const int qa = i >= 1 ? qa_next : 0;
        uint32_t wpack = 0;  // DNA: the 4 scores of the query letter, one byte each
        const int8_t *wrow = sW + qa * A;
        if constexpr (DNA) wpack = *reinterpret_cast<const uint32_t *>(wrow);
        if (i >= 1) {
            // the window moves one column right per row
#pragma unroll
            for (int k = 0; k < W - 1; k++) tw[k] = tw[k + 1];
            tw[W - 1] = tn_next;
            qa_next = qletter(i + 1);
            tn_next = tletter(i + 1);
        }
        int holeft = negho, eleft = kNegB;
        typename DirWord<W>::T dw;
        zero<W>(dw);
        int row_hit = -1;
        int rmax = kNegB;  // REV: the row's maximum (no anchored path scores above target)
        // rows whose band cells all lie inside the rectangle (most of them,
        // but not the last, which holds the final cell): no boundary tests
        // per cell.  The callers pass wb == W (a band wider than the
        // provable one is still exact), so no cell lies past the band.
        const bool interior = i >= 1 && i < s.rows + (REV ? 1 : 0) && i + dlo >= 1 && i + dlo + wb - 1 <= s.cols;
        if (interior) {
#pragma unroll
            for (int k = 0; k < W; k++) {
                const int houp = k + 1 < W ? Hp[k + 1] : negho;  // H(i-1, j) - O: where F opens
                const int fup = k + 1 < W ? Fp[k + 1] : kNegB;
                const int F = max(houp, fup - X);
                const int E = max(holeft, eleft - X);
                int w;
                if constexpr (DNA) w = (int)(int8_t)(uint8_t)(wpack >> tw[k]);
                else w = wrow[tw[k]];
                const int hdg = Hp[k] + w + O;  // H(i-1, j-1) + W
                const int H = max(hdg, max(E, F));
                if constexpr (REV) {
                    rmax = max(rmax, H);
                } else {
                    uint32_t &bw = nib_word<W>(dw, k);
                    const int sh = 4 * (k & 7);
                    or_if_ne(bw, H, hdg, 1u << sh);
                    or_if_ne(bw, H, E, 2u << sh);
                    or_if_ne(bw, E, holeft, 4u << sh);
                    or_if_ne(bw, F, houp, 8u << sh);
                }
                const int ho = H - O;
                Hp[k] = ho;
                Fp[k] = F;
                holeft = ho;
                eleft = E;
            }
            if constexpr (REV) {
                if (rmax == target) {
                    // the row reaches target: its first cell that does
#pragma unroll
                    for (int k = W - 1; k >= 0; k--)
                        if (Hp[k] == target - O) row_hit = i + dlo + k;
                }
            }
        } else {
#pragma unroll
        for (int k = 0; k < W; k++) {
            const int j = i + dlo + k;
            const bool valid = k < wb && j >= 0 && j <= s.cols;
            const int houp = k + 1 < W ? Hp[k + 1] : negho;
            const int fup = k + 1 < W ? Fp[k + 1] : kNegB;
            int F = kNegB, hdg = kNegB, E = kNegB, H;
            bool fopen = false, eopen = false;
            if (i >= 1) {
                F = max(houp, fup - X);
                fopen = F == houp;
            }
            if (i >= 1 && j >= 1 && valid) {
                int w;
                if constexpr (DNA) w = (int)(int8_t)(uint8_t)(wpack >> tw[k]);
                else w = wrow[tw[k]];
                hdg = Hp[k] + w + O;
            }
            if (j >= 1) {
                E = max(holeft, eleft - X);
                eopen = E == holeft;
            }
            H = max(hdg, max(E, F));
            if (i == 0 && j == 0) H = 0;
            if (!valid || H < kNegBHalf) {
                H = kNegB;
                E = kNegB;
                F = kNegB;
            }
            if constexpr (REV) {
                if (i >= 1 && j >= 1 && H == target && row_hit < 0) row_hit = j;
            } else {
                const bool diag = i >= 1 && j >= 1 && hdg > kNegBHalf && H == hdg;
                put_nib<W>(dw, k, (diag ? 0u : 1u) | (H != E ? 2u : 0u) | (eopen ? 0u : 4u) | (fopen ? 0u : 8u));
                if (i == s.rows && j == s.cols) fin = H;
            }
            // this row's value becomes the next row's "previous row"
            Hp[k] = H - O;
            Fp[k] = F;
            holeft = H - O;
            eleft = E;
        }
        }
        if constexpr (REV) {
            if (row_hit >= 0 && row_hit < best_j) {
                best_j = row_hit;
                best_i = i;
            }
            // no later row can reach a column <= best_j inside the band
            if (best_j != INT_MAX && i + 1 + dlo >= best_j) break;
        } else {
            *drow = dw;
            drow += rstride;
        }
    }
    if constexpr (REV) {
        *out_i = best_i;
        *out_j = best_j;
        return best_j != INT_MAX;
    } else {
        *final_h = fin;
        return true;
    }
}

// Walks the decision nibbles from (la, lb) back to (0, 0).  With WRITE the
// runs go to out[0..nr) in forward order; otherwise the first `keep` runs
// found (the CIGAR's last ones) go to out[0..keep) in the order found.
// Returns the run count or -1.  Rows are STRIDE words of the template apart.
template <int W, bool WRITE, int STRIDE = 32>
__device__ int band_walk(const typename DirWord<W>::T *dirs, int la, int lb, int dlo, int wb, uint32_t *out, int nr,
                         int keep = 0) {
    int i = la, j = lb, state = 0, cur = -1, len = 0, runs = 0, guard = 2 * (la + lb) + 4;
    // the walk moves up at most one row per step: it holds the current row's
    // word and the one above, loaded when the row before it was entered
    typename DirWord<W>::T word = dirs[(long long)la * STRIDE], above;
    if (la > 0) above = dirs[(long long)(la - 1) * STRIDE];
    else zero<W>(above);
    int row = la;
    while ((i > 0 || j > 0) && guard-- > 0) {
        const int k = j - i - dlo;
        if (i < 0 || j < 0 || k < 0 || k >= wb) return -1;
        if (i != row) {
            word = above;
            row = i;
            if (i > 0) above = dirs[(long long)(i - 1) * STRIDE];
        }
        const uint32_t nib = get_nib<W>(word, k);
        int op;
        if (state == 0 && !(nib & 1)) {
            op = GSW_CIGAR_M;  // preference: the diagonal, then E, then F
            i--;
            j--;
        } else {
            if (state == 0) state = (nib & 2) ? 2 : 1;
            if (state == 1) {
                op = GSW_CIGAR_D;
                state = (nib & 4) ? 1 : 0;
                j--;
            } else {
                op = GSW_CIGAR_I;
                state = (nib & 8) ? 2 : 0;
                i--;
            }
        }
        if (op == cur) {
            len++;
        } else {
            if (len) {
                if (WRITE) out[nr - 1 - runs] = ((uint32_t)len << 4) | (uint32_t)cur;
                else if (runs < keep) out[runs] = ((uint32_t)len << 4) | (uint32_t)cur;
                runs++;
            }
            cur = op;
            len = 1;
        }
    }
    if (i != 0 || j != 0) return -1;
    if (len) {
        if (WRITE) out[nr - 1 - runs] = ((uint32_t)len << 4) | (uint32_t)cur;
        else if (runs < keep) out[runs] = ((uint32_t)len << 4) | (uint32_t)cur;
        runs++;
    }
    return runs;
}

struct BandLaunch {
    BatchView b;
    Scoring sc;
    const int32_t *order;
    const int32_t *var_start;  // per class
    int32_t *head;             // per class task counters
    void *scratch;             // per warp: (maxrows + 1) * 32 direction words of the class width
    int64_t scratch_words;     // per warp, in 32-bit words
};

// Banded global DP, walk and CIGAR output of one pair in the narrowest
// template that holds its band (WT cells per row).  The decision words of
// the warp's lanes are interleaved row by row in the class's layout (W cells
// per lane and row) whatever template each lane takes, so the rows of lanes
// with different templates never overlap.
template <int W, int WT>
__device__ void band_trace(const BatchView &b, const Scoring &sc, gsw_result *rp, const BandSeq &s, int dlo, int wb,
                           int s1, const int8_t *sW, uint32_t *warp_scratch, int lane) {
    using DW = typename DirWord<WT>::T;
    constexpr int RSTRIDE = 32 * (W / WT);  // a row of 32 lanes of W/8 words, in DW units
    DW *dirs = reinterpret_cast<DW *>(warp_scratch + (size_t)lane * (W / 8));
    const int la = s.rows, lb = s.cols;
    wb = WT;  // the band widened to the template: still exact, no per-cell width test
    int fin = 0, di, dj;
    if (sc.dna4) band_dp<WT, false, true>(s, dlo, wb, sW, sc.A, sc.O, sc.X, 0, dirs, &di, &dj, &fin, RSTRIDE);
    else band_dp<WT, false, false>(s, dlo, wb, sW, sc.A, sc.O, sc.X, 0, dirs, &di, &dj, &fin, RSTRIDE);
    if (fin != s1) {
        rp->flags |= kResInternal;
        return;
    }
    // one walk keeps up to kKeep runs (true reads have a few); a CIGAR with
    // more is walked a second time, into its reserved words
    constexpr int kKeep = 16;
    uint32_t kept[kKeep];
    const int nr = band_walk<WT, false, RSTRIDE>(dirs, la, lb, dlo, wb, kept, 0, kKeep);
    if (nr < 0) {
        rp->flags |= kResInternal;
        return;
    }
    const unsigned long long off = atomicAdd(b.cigar_cursor, (unsigned long long)nr);
    if ((long long)(off + nr) > b.cigar_cap) {
        rp->flags |= GSW_RES_CIGAR_SPACE;
        rp->cigar_len = -nr;
        rp->cigar_off = -1;
        return;
    }
    if (nr <= kKeep) {
        for (int q = 0; q < nr; q++) b.cigar[off + q] = kept[nr - 1 - q];
    } else {
        band_walk<WT, true, RSTRIDE>(dirs, la, lb, dlo, wb, b.cigar + off, nr);
    }
    rp->cigar_len = nr;
    rp->cigar_off = (int64_t)off;
}

template <int W>
__device__ void band_pair(const BandLaunch &L, int p, const int8_t *sW, uint32_t *warp_scratch, int lane) {
    const BatchView &b = L.b;
    const Scoring &sc = L.sc;
    gsw_result *rp = b.res + p;
    const int s1 = rp->score1, eq = rp->read_end1, et = rp->ref_end1;
    const uint8_t *qp = b.q + b.q_off[p];
    const uint8_t *tp = b.t + b.t_off[p];
    int bq = rp->read_begin1, bt = rp->ref_begin1;
    if (bq < 0 || bt < 0) {
        // reverse band: G diagonals above the main one (target letters
        // against gaps), Gn below (query letters against gaps)
        const int G = reverse_gap_bound(eq, s1, sc);
        const int Gn = reverse_gap_bound_rows(eq, s1, sc);
        if (G < 0 || G + Gn + 1 > W) {  // the plan's class holds the reverse band
            rp->flags |= kResInternal;
            return;
        }
        BandSeq s{qp + eq, -1, eq + 1, tp + et, -1, reverse_window(eq, et, s1, sc)};
        int bi, bj, dummy;
        // (widened to the template's W diagonals: still exact)
        const bool ok = sc.dna4 ? band_dp<W, true, true>(s, -Gn, W, sW, sc.A, sc.O, sc.X, s1, nullptr, &bi, &bj, &dummy)
                                : band_dp<W, true, false>(s, -Gn, W, sW, sc.A, sc.O, sc.X, s1, nullptr, &bi, &bj, &dummy);
        if (!ok) {
            rp->flags |= kResInternal;
            return;
        }
        bq = eq - (bi - 1);
        bt = et - (bj - 1);
        rp->read_begin1 = bq;
        rp->ref_begin1 = bt;
    }
    if (!(b.flags & GSW_CIGAR)) return;
    const int la = eq - bq + 1, lb = et - bt + 1;
    const int w = band_halfwidth(la, lb, s1, sc);
    const int delta = lb - la;
    const int dlo = max(min(0, delta) - w, -la), dhi = min(max(0, delta) + w, lb);
    const int wb = dhi - dlo + 1;
    if (wb > W) {
        rp->flags |= kResPendingTrace;  // the warp traceback takes it
        return;
    }
    // the traceback band is usually much narrower than the reverse band that
    // put the pair in this class
    const BandSeq s{qp + bq, 1, la, tp + bt, 1, lb};
    if (wb <= 8) band_trace<W, 8>(b, sc, rp, s, dlo, wb, s1, sW, warp_scratch, lane);
    else if constexpr (W >= 16) {
        if (wb <= 16) band_trace<W, 16>(b, sc, rp, s, dlo, wb, s1, sW, warp_scratch, lane);
        else if constexpr (W >= 32) band_trace<W, 32>(b, sc, rp, s, dlo, wb, s1, sW, warp_scratch, lane);
    }
}

template <int W, int CLS>
__global__ void __launch_bounds__(kBBlock) k_band(BandLaunch L) {
    __shared__ __align__(4) int8_t sW[kMaxAlpha * kMaxAlpha];
    for (int i = threadIdx.x; i < L.sc.A * L.sc.A; i += blockDim.x) sW[i] = L.sc.W[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (kBBlock / 32) + warp;
    uint32_t *warp_scratch = reinterpret_cast<uint32_t *>(L.scratch) + (size_t)gwarp * L.scratch_words;
    const int first = L.var_start[CLS], last = L.var_start[CLS + 1];
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&L.head[CLS], 1);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        const int idx = first + t * 32 + lane;
        if (first + t * 32 >= last) break;
        if (idx < last) band_pair<W>(L, L.order[idx], sW, warp_scratch, lane);
        __syncwarp();
    }
}

}  // namespace

int band_block_threads() { return kBBlock; }

// Resident blocks per SM of each class's kernel (width 8, 16, 32).
static void band_occupancy(int occ[3]) {
    occ[0] = occ[1] = occ[2] = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_band<8, 0>, kBBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_band<16, 1>, kBBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_band<32, 2>, kBBlock, 0);
    for (int c = 0; c < 3; c++) occ[c] = std::max(1, occ[c]);
}

BandGrids band_grids(int rows_cap, int sms, size_t budget_bytes) {
    int occ[3];
    band_occupancy(occ);
    BandGrids g;
    size_t total = 0;
    for (int c = 0; c < 3; c++) {
        // a warp's rows: (rows_cap + 1) x 32 lanes x W/8 words
        g.words[c] = (int64_t)(rows_cap + 1) * 32 * ((8 << c) / 8);
        g.grid[c] = sms * occ[c];
        total += (size_t)g.grid[c] * (kBBlock / 32) * (size_t)g.words[c] * sizeof(uint32_t);
    }
    const double scale = total > budget_bytes && total > 0 ? (double)budget_bytes / (double)total : 1.0;
    size_t off = 0;
    for (int c = 0; c < 3; c++) {
        g.grid[c] = std::max(1, (int)(g.grid[c] * scale));
        g.off[c] = off;
        off += (size_t)g.grid[c] * (kBBlock / 32) * (size_t)g.words[c] * sizeof(uint32_t);
        off = (off + 255) & ~(size_t)255;
    }
    g.total_bytes = off;
    return g;
}

cudaError_t launch_band(const BatchView &b, const Scoring &sc, const PlanBuffers &pb, void *scratch,
                        const BandGrids &g, cudaStream_t st, const BandStreams &aux) {
    BandLaunch L;
    L.b = b;
    L.sc = sc;
    L.order = pb.order;
    L.var_start = pb.var_start;
    L.head = pb.task_lo;  // reused as per-class counters (zeroed below)
    cudaMemsetAsync(pb.task_lo, 0, sizeof(int32_t) * kNumVariants, st);
    // the three classes run side by side (each its own scratch): the widest
    // (slowest per pair) on the calling stream, the others on two auxiliary
    // streams forked and joined by events, so a class's tail overlaps the others
    cudaEventRecord(aux.fork, st);
    cudaStreamWaitEvent(aux.s[0], aux.fork, 0);
    cudaStreamWaitEvent(aux.s[1], aux.fork, 0);
    const cudaStream_t on[3] = {aux.s[1], aux.s[0], st};
    for (int c = 2; c >= 0; c--) {
        L.scratch = static_cast<uint8_t *>(scratch) + g.off[c];
        L.scratch_words = g.words[c];
        if (c == 2) k_band<32, 2><<<g.grid[2], kBBlock, 0, on[2]>>>(L);
        else if (c == 1) k_band<16, 1><<<g.grid[1], kBBlock, 0, on[1]>>>(L);
        else k_band<8, 0><<<g.grid[0], kBBlock, 0, on[0]>>>(L);
    }
    cudaEventRecord(aux.join[0], aux.s[0]);
    cudaEventRecord(aux.join[1], aux.s[1]);
    cudaStreamWaitEvent(st, aux.join[0], 0);
    cudaStreamWaitEvent(st, aux.join[1], 0);
    return cudaGetLastError();
}

}  // namespace gsw
