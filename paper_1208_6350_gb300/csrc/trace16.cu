// Traceback of pairs with wide bands in 16-bit lanes: the global Gotoh DP
// between begin and end ("Algorithm and implementation", item (1): the banded
// SW whose band the begin and end define yields the CIGAR), computed over the
// whole rectangle q[begin..end] x t[begin..end], strip after strip of 64 to
// 256 query rows, when every value of it fits a biased 16-bit lane.
//
// The rectangle contains every band, and the traceback over it is the
// oracle's own definition (the full-rectangle DP), so the CIGAR is the
// canonical one.  For random local alignments (bands of hundreds of
// diagonals) the provable band covers most of the rectangle anyway; the
// rectangle in the folded ring of the fill (fill.cu) costs about a quarter of
// the instructions per cell of the 32-bit anti-diagonal kernel.
//
// Layout: a group of 8 lanes per pair; lane k holds R 32-bit words, word r
// packing row k*R + r (bits 0-15) and row S + k*R + r (bits 16-31), S = 8R,
// each as value + 0x8000.  Step s computes target column s - k of the low
// half and column s - k - 8 of the high half; the bottom row (H, F) goes down
// the ring by a shuffle, lane 7's low half wrapping to lane 0's high half.
// Boundaries are those of the oracle's recurrences with H(0,0) = 0 and -inf
// outside: H(0,j) = -(O + (j-1)X), H(i,0) = -(O + (i-1)X), E(i,1) = H(i,0) - O,
// F(1,j) = H(0,j) - O.  A region taller than a strip runs strip after strip:
// lane 7's high half (the strip's last row) leaves H and F(next row) per
// column in a ping-pong buffer, which the next strip's lane 0 reads in place
// of the top boundary, one block of 8 columns ahead.
//
// Per cell (i, j) 4 bits: bit 0 H != H(i-1,j-1) + W; bit 1 H != E(i,j);
// bit 2 E(i,j+1) != H(i,j) - O (the horizontal gap through (i,j+1) extends
// rather than opens at (i,j)); bit 3 F(i+1,j) != H(i,j) - O.  Bits 2-3
// describe the cell's successors because the step computes E(i,j+1) and
// F(i+1,j) from this cell; the walk reaches (i,j) from (i,j+1) or (i+1,j) and
// needs exactly those.  A lane packs its 2R nibbles of a step into R/4 words
// (low-half nibbles in bits 0-15, high-half ones in bits 16-31); the group
// writes the step's 8 x R/4 words contiguously (word q of lane k at
// [s][q][k]).
//
// The walk from (la, lb) runs on all 8 lanes of the group in lockstep over
// tiles of decision words staged in the (then unused) profile shared memory.
#include "gsw_impl.cuh"

#include <algorithm>
#include <climits>

namespace gsw {
namespace {

constexpr int kT16Block = 128;
constexpr int kP = kT16P;

// per-lane profile words: DNA a low-letter and a high-letter table (4 + 4
// letters x R words, plain integers w and w * 65536: H(i-1,j-1) + W is one
// 3-input add); other alphabets one table of A letters x R words with both
// halves' scores (16-bit two's-complement halves)
__host__ __device__ inline int t16_prof_words(int R, bool dna, int A) { return dna ? 8 * R : A * R; }

// word (table entry c, row r) of lane l inside a warp's region: lane-minor
// 16-byte vectors, so the 8 lanes of a quarter warp cover all 32 banks
template <int R>
__device__ __forceinline__ int t16_pidx(int c, int r, int l) {
    return ((c * (R / 4) + r / 4) * 32 + l) * 4 + (r & 3);
}

template <int R>
__device__ __forceinline__ void t16_load(const uint32_t *base, int c, int l, uint32_t (&w)[R]) {
#pragma unroll
    for (int r = 0; r < R; r += 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(base + t16_pidx<R>(c, r, l));
        w[r] = v.x;
        w[r + 1] = v.y;
        w[r + 2] = v.z;
        w[r + 3] = v.w;
    }
}

// biased H(i, 0) (and H(0, i)): -(O + (i-1)X), H(0,0) = 0
__device__ __forceinline__ uint32_t t16_edge(int i, int O, int X) {
    return (uint32_t)(0x8000 - (i == 0 ? 0 : O + (i - 1) * X)) & 0xFFFFu;
}

template <int R, bool DNA>
struct T16Runner {
    static constexpr int S = kP * R;
    static constexpr int SS = 2 * S;  // rows of a strip
    static constexpr int Q = R / 4;

    const uint8_t *qs;  // query region, row i (0-based) at qs[i]
    const uint8_t *ts;  // target region, column j (0-based) at ts[j]
    int la, lb, A, O, X, k, src, gbase, st;
    unsigned gmask;
    uint32_t *psm, *dirs, *fin_words;
    const uint32_t *bin;  // previous strip's last row: H | F(next row) << 16 per column
    uint32_t *bout;
    int lane;
    uint32_t kO, kXm, hb0, stepX;
    uint32_t H[R], E[R];
    uint32_t xh, xf, hdiag, b_cur, b_nxt;
    int nal, nah;
    // the cell (la, lb): strip, step, lane, word and half holding it
    int st_fin, s_fin, k_fin, r_fin, h_fin;
    int fh;

    __device__ __forceinline__ void init(const uint8_t *qs_, int la_, const uint8_t *ts_, int lb_, const Scoring &sc,
                                         uint32_t *psm_, uint32_t *fin_words_, int k_, int lane_, unsigned gmask_,
                                         int gbase_) {
        qs = qs_;
        la = la_;
        ts = ts_;
        lb = lb_;
        A = sc.A;
        O = sc.O;
        X = sc.X;
        k = k_;
        lane = lane_;
        gmask = gmask_;
        gbase = gbase_;
        src = gbase_ + ((k_ + kP - 1) & (kP - 1));
        psm = psm_;
        fin_words = fin_words_;
        kO = (uint32_t)(-O * 65537);
        kXm = ((uint32_t)(-X) & 0xFFFFu) * 0x10001u;
        stepX = (uint32_t)X * 0x10001u;
        st_fin = (la - 1) / SS;
        const int ri = la - 1 - st_fin * SS, hh = ri >= S ? 1 : 0, rr = ri - hh * S;
        k_fin = rr / R;
        r_fin = rr - k_fin * R;
        h_fin = hh;
        s_fin = lb - 1 + k_fin + hh * kP;
        fh = INT_MIN;
        // every lane has read its old op words (the walk of the group's
        // previous pair) before the lane holding (la, lb) overwrites them
        __syncwarp(gmask);
    }

    // Starts strip st_ (rows st_*SS ..): its profile, the left boundary of
    // its rows, and the row above it (the top boundary for strip 0, else the
    // previous strip's last row from bin_).
    __device__ __forceinline__ void begin(const Scoring &sc, int st_, uint32_t *dirs_, const uint32_t *bin_,
                                          uint32_t *bout_) {
        st = st_;
        dirs = dirs_;
        bin = bin_;
        bout = bout_;
        const int i0 = st * SS;
        // profile of the lane's rows (rows past la score 0)
#pragma unroll 1
        for (int r = 0; r < R; r++) {
            const int ilo = i0 + k * R + r, ihi = i0 + S + k * R + r;
            const int qlo = ilo < la ? min((int)qs[ilo], A - 1) : -1;
            const int qhi = ihi < la ? min((int)qs[ihi], A - 1) : -1;
            if constexpr (DNA) {
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int wl = qlo >= 0 ? sc.W[qlo * 4 + a] : 0;
                    const int wh = qhi >= 0 ? sc.W[qhi * 4 + a] : 0;
                    psm[t16_pidx<R>(a, r, lane)] = (uint32_t)wl;
                    psm[t16_pidx<R>(4 + a, r, lane)] = (uint32_t)(wh * 65536);
                }
            } else {
                for (int a = 0; a < A; a++) {
                    const int wl = qlo >= 0 ? sc.W[qlo * A + a] : 0;
                    const int wh = qhi >= 0 ? sc.W[qhi * A + a] : 0;
                    psm[t16_pidx<R>(a, r, lane)] = ((uint32_t)wl & 0xFFFFu) | (((uint32_t)wh & 0xFFFFu) << 16);
                }
            }
        }
        // left boundary: H(i, 0) and E(i, 1) = H(i, 0) - O of the lane's rows
        hb0 = t16_edge(i0 + k * R + 1, O, X) | (t16_edge(i0 + S + k * R + 1, O, X) << 16);
#pragma unroll
        for (int r = 0; r < R; r++) {
            H[r] = hb0 - (uint32_t)r * stepX;
            E[r] = H[r] + kO;
        }
        // the row above the lane's first rows at column 0 (the diagonal of
        // lane 1's first column; later lanes get it down the ring)
        xh = t16_edge(i0 + k * R, O, X) | (t16_edge(i0 + S + k * R, O, X) << 16);
        xf = 0;
        hdiag = t16_edge(i0, O, X) * 0x10001u;  // lane 0: H(i0, 0), the diagonal of its first cell
        nal = (k == 0) ? min((int)ts[0], A - 1) : 0;
        nah = 0;
        b_cur = 0;
        b_nxt = 0;
        if (st > 0) prefetch(0);
    }

    // The previous strip's row for columns [s0, s0 + 8): lane k loads column
    // s0 + k, lane 0 takes each by a shuffle in its step
    __device__ __forceinline__ void prefetch(int s0) {
        const int j = s0 + k;
        b_nxt = j < lb ? bin[j] : 0u;
    }

    template <bool CHECKED>
    __device__ __forceinline__ void step(const int s) {
        const int jlo = s - k;
        const int jhi = jlo - kP;
        // lane 0's low half: the row above the strip at column s (the top
        // boundary H(0, s+1) for strip 0 and past the last column)
        uint32_t tlo = (uint32_t)(0x8000 - O - s * X) & 0xFFFFu;
        uint32_t flo = (tlo - (uint32_t)O) & 0xFFFFu;
        if (st > 0) {
            if ((s & (kP - 1)) == 0) {
                b_cur = b_nxt;
                prefetch(s + kP);
            }
            const uint32_t w = __shfl_sync(gmask, b_cur, gbase + (s & (kP - 1)));
            if (s < lb) {
                tlo = w & 0xFFFFu;
                flo = w >> 16;
            }
        }
        // lane 0's high half continues lane 7's low half
        const uint32_t hin = k == 0 ? ((xh << 16) | tlo) : xh;
        const uint32_t fin = k == 0 ? ((xf << 16) | flo) : xf;
        const int al = nal, ah = nah;
        {
            const int j1 = jlo + 1;
            if constexpr (CHECKED) {
                nal = (j1 >= 0 && j1 < lb) ? min((int)ts[j1], A - 1) : 0;
                nah = (j1 - kP >= 0 && j1 - kP < lb) ? min((int)ts[j1 - kP], A - 1) : 0;
            } else {
                nal = min((int)ts[j1], A - 1);
                nah = min((int)ts[j1 - kP], A - 1);
            }
        }
        uint32_t pw[R], ph[R];
        if constexpr (DNA) {
            t16_load<R>(psm, al, lane, pw);
            t16_load<R>(psm, 4 + ah, lane, ph);
        } else {
            t16_load<R>(psm, al, lane, pw);
            t16_load<R>(psm, ah, lane, ph);
        }
        uint32_t diag = hdiag;
        hdiag = hin;
        uint32_t f = fin;
        uint32_t acc[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) acc[q] = 0;
        constexpr uint32_t ONE2 = 0x00010001u;
#pragma unroll
        for (int r = 0; r < R; r++) {
            uint32_t hdg;
            if constexpr (DNA) hdg = diag + pw[r] + ph[r];
            else hdg = __viaddmax_u16x2(diag, (pw[r] & 0x0000FFFFu) | (ph[r] & 0xFFFF0000u), 0u);
            const uint32_t e = E[r];
            const uint32_t h = __vmaxu2(hdg, __vmaxu2(e, f));
            const uint32_t ho = h + kO;
            const uint32_t e2 = __viaddmax_u16x2(e, kXm, ho);
            const uint32_t f2 = __viaddmax_u16x2(f, kXm, ho);
            // each difference is >= 0 in both halves: no borrow between them
            const uint32_t nib = __vminu2(h - hdg, ONE2) + 2u * __vminu2(h - e, ONE2) +
                                 4u * __vminu2(e2 - ho, ONE2) + 8u * __vminu2(f2 - ho, ONE2);
            acc[r / 4] += nib << (4 * (r & 3));
            diag = H[r];
            H[r] = h;
            E[r] = e2;
            f = f2;
        }
        uint32_t *dst = dirs + (size_t)s * (Q * kP) + k;
#pragma unroll
        for (int q = 0; q < Q; q++) dst[q * kP] = acc[q];
        // lane 7 holds the strip's last row: the next strip's top
        if (bout && k == kP - 1 && jhi >= 0 && jhi < lb) bout[jhi] = (H[R - 1] >> 16) | (f & 0xFFFF0000u);
        if constexpr (CHECKED) {
            // before a half's first column its rows hold the left boundary
            if (jhi < 0) {
                const uint32_t keep = jlo >= 0 ? 0x0000FFFFu : 0u;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const uint32_t hb = hb0 - (uint32_t)r * stepX;
                    H[r] = (H[r] & keep) | (hb & ~keep);
                    E[r] = (E[r] & keep) | ((hb + kO) & ~keep);
                }
            }
        }
        // the lane holding (la, lb) parks its words (a select by a run-time
        // row would put H in local memory)
        if (st == st_fin && s == s_fin && k == k_fin) {
#pragma unroll
            for (int r = 0; r < R; r++) fin_words[r] = H[r];
        }
        xh = __shfl_sync(gmask, H[R - 1], src);
        xf = __shfl_sync(gmask, f, src);
    }

    // the strip over every column: start-up (some half before its first
    // column), steady (every column in range), drain (columns past lb)
    __device__ __forceinline__ void run() {
        const int nsteps = t16_steps(lb);
        const int s_steady = 2 * kP - 1;
        const int s_drain = max(s_steady, lb - 1);
        int s = 0;
#pragma unroll 1
        for (; s < s_steady; s++) step<true>(s);
#pragma unroll 1
        for (; s < s_drain; s++) step<false>(s);
#pragma unroll 1
        for (; s < nsteps; s++) step<true>(s);
        // the next strip reads this one's boundary row, the walk its words
        __syncwarp(gmask);
    }

    // H(la, lb), once its strip has run
    __device__ __forceinline__ int final_h() const {
        return (int)((fin_words[r_fin] >> (16 * h_fin)) & 0xFFFFu) - 0x8000;
    }
};

// Appends `n` ops `op` to the run-length walk (runs in reverse order).
__device__ __forceinline__ void t16_emit(int op, int n, int &cur, int &len, int &runs, uint32_t *ops, bool writer) {
    if (op == cur) {
        len += n;
        return;
    }
    if (len) {
        if (writer) ops[runs] = ((uint32_t)len << 4) | (uint32_t)cur;
        runs++;
    }
    cur = op;
    len = n;
}

// Walk of one pair from (la, lb) over the group's direction words; all 8
// lanes take the same path, lane 0 writes the runs.  Returns the run count,
// or -1 if the walk left the rectangle (never for consistent words).
template <int R>
__device__ __forceinline__ int t16_walk(const uint32_t *dirs, uint32_t *stage, int tile_steps, int la, int lb, int k,
                                        unsigned gmask, uint32_t *ops) {
    constexpr int S = kP * R;
    constexpr int SS = 2 * S;
    constexpr int Q = R / 4;
    const int nsteps = t16_steps(lb);
    int i = la, j = lb, mode = 0, cur = -1, len = 0, runs = 0;
    int tile_lo = INT_MAX;
    const bool writer = k == 0;
    int guard = la + lb + 2;
    while (i > 0 && j > 0 && guard-- > 0) {
        const int st = (i - 1) / SS;
        const int ri = i - 1 - st * SS;
        const int hh = ri >= S ? 1 : 0;
        const int rr = ri - hh * S;
        const int kk = rr / R, rs = rr - kk * R;
        // step index over the strips laid end to end: it never increases
        // along the walk, so the group stages the tile ending at it
        const int s = st * nsteps + j - 1 + kk + hh * kP;
        if (s < tile_lo) {
            // 16-byte asynchronous copies, all in flight at once (the words
            // were just written: L2), then one wait
            __syncwarp(gmask);
            tile_lo = max(0, s - tile_steps + 1);
            const int n4 = (s - tile_lo + 1) * (Q * kP) / 4;
            const uint4 *from = reinterpret_cast<const uint4 *>(dirs + (size_t)tile_lo * (Q * kP));
            for (int w = k; w < n4; w += kP) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(stage + 4 * w);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(from + w) : "memory");
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncwarp(gmask);
        }
        const uint32_t nib = (stage[((s - tile_lo) * Q + (rs >> 2)) * kP + kk] >> (16 * hh + 4 * (rs & 3))) & 15u;
        if (mode == 1) {  // in a horizontal gap that reached (i, j + 1)
            if (nib & 4u) {
                t16_emit(GSW_CIGAR_D, 1, cur, len, runs, ops, writer);
                j--;
                continue;
            }
            mode = 0;
        } else if (mode == 2) {  // in a vertical gap that reached (i + 1, j)
            if (nib & 8u) {
                t16_emit(GSW_CIGAR_I, 1, cur, len, runs, ops, writer);
                i--;
                continue;
            }
            mode = 0;
        }
        if (!(nib & 1u)) {
            t16_emit(GSW_CIGAR_M, 1, cur, len, runs, ops, writer);
            i--;
            j--;
        } else if (!(nib & 2u)) {
            t16_emit(GSW_CIGAR_D, 1, cur, len, runs, ops, writer);
            j--;
            mode = 1;
        } else {
            t16_emit(GSW_CIGAR_I, 1, cur, len, runs, ops, writer);
            i--;
            mode = 2;
        }
    }
    if (i < 0 || j < 0 || (i > 0 && j > 0)) return -1;
    // the boundary row or column: gaps to the origin
    if (i > 0) t16_emit(GSW_CIGAR_I, i, cur, len, runs, ops, writer);
    if (j > 0) t16_emit(GSW_CIGAR_D, j, cur, len, runs, ops, writer);
    if (len) {
        if (writer) ops[runs] = ((uint32_t)len << 4) | (uint32_t)cur;
        runs++;
    }
    return runs;
}

template <int R, bool DNA>
__global__ void __launch_bounds__(kT16Block) k_trace16(BatchView b, Scoring sc, T16Scratch ts, int cls) {
    extern __shared__ __align__(16) uint32_t t16_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / kP, k = lane & (kP - 1), gbase = lane & ~(kP - 1);
    const unsigned gmask = ((1u << kP) - 1u) << gbase;
    const int pwords = t16_prof_words(R, DNA, sc.A);
    uint32_t *psm = t16_smem + (size_t)warp * 32 * pwords;
    // after the fills, group g stages its walk tiles in quarter g of the region
    uint32_t *stage = psm + (size_t)g * kP * pwords;
    const int tile_steps = pwords / (R / 4);
    const int gwarp = blockIdx.x * (kT16Block / 32) + warp;
    const size_t gid = (size_t)gwarp * (32 / kP) + g;
    const int v = cls - kTraceT16First;
    const int64_t dir_words = ts.dir_words[v];
    uint32_t *dirs = ts.dirs + gid * dir_words;
    uint32_t *ops = ts.ops + gid * ts.op_words;
    const int first = ts.var_start[cls], last = ts.var_start[cls + 1];
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&ts.head[cls], 1);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        const int base = first + t * (32 / kP);
        if (base >= last) break;
        const int idx = base + g;
        int p = -1, la = 0, lb = 0, score1 = 0;
        if (idx < last) {
            p = ts.order[idx];
            const gsw_result &rr = b.res[p];
            score1 = rr.score1;
            const int flags = rr.flags, qb = rr.read_begin1, tb = rr.ref_begin1;
            la = rr.read_end1 - qb + 1;
            lb = rr.ref_end1 - tb + 1;
            const bool fits = score1 > 0 && (flags & kResPendingTrace) && !(flags & kResInternal) && qb >= 0 &&
                              tb >= 0 && la >= 1 && lb >= 1 && lb <= kT16MaxCols &&
                              t16_need_words(la, lb, v) <= dir_words && (long long)la + lb + 2 <= ts.op_words;
            if (!fits) {
                if (k == 0 && score1 > 0 && (flags & kResPendingTrace)) b.res[p].flags |= kResInternal;
                p = -1;
            }
        }
        int fh = INT_MIN;
        if (p >= 0) {
            // each lane builds and reads only its own profile words
            T16Runner<R, DNA> run;
            run.init(b.q + b.q_off[p] + b.res[p].read_begin1, la, b.t + b.t_off[p] + b.res[p].ref_begin1, lb, sc,
                     psm, ops, k, lane, gmask, gbase);
            const int nst = t16_strips(la, v);
            const size_t strip_words = (size_t)t16_steps(lb) * (R / 4) * kP;
            uint32_t *bnd0 = dirs + strip_words * nst, *bnd1 = bnd0 + ((lb + 3) & ~3);
#pragma unroll 1
            for (int st = 0; st < nst; st++) {
                const uint32_t *bin = st == 0 ? nullptr : ((st & 1) ? bnd0 : bnd1);
                uint32_t *bout = st + 1 < nst ? ((st & 1) ? bnd1 : bnd0) : nullptr;
                run.begin(sc, st, dirs + strip_words * st, bin, bout);
                run.run();
            }
            fh = run.final_h();
        }
        __syncwarp();  // every group's fill is done: the profile region is free
        int nr = -1;
        if (p >= 0 && fh == score1) {
            // the dirs the group wrote are visible to its lanes after the warp barrier
            nr = t16_walk<R>(dirs, stage, tile_steps, la, lb, k, gmask, ops);
        }
        if (p >= 0) {
            __syncwarp(gmask);
            if (nr < 0) {
                if (k == 0) b.res[p].flags |= kResInternal;
            } else {
                unsigned long long off = 0;
                if (k == 0) off = atomicAdd(b.cigar_cursor, (unsigned long long)nr);
                off = __shfl_sync(gmask, off, gbase);
                gsw_result *rp = b.res + p;
                if ((long long)(off + nr) > b.cigar_cap) {
                    if (k == 0) {
                        rp->flags |= GSW_RES_CIGAR_SPACE;
                        rp->cigar_len = -nr;
                        rp->cigar_off = -1;
                        rp->flags &= ~kResPendingTrace;
                    }
                } else {
                    for (int x = k; x < nr; x += kP) b.cigar[off + x] = ops[nr - 1 - x];
                    if (k == 0) {
                        rp->cigar_len = nr;
                        rp->cigar_off = (int64_t)off;
                        rp->flags &= ~kResPendingTrace;
                    }
                }
            }
        }
        __syncwarp();  // the next task rebuilds the profile region
    }
}

template <int R, bool DNA>
size_t t16_smem_bytes(const Scoring &sc) {
    return (size_t)(kT16Block / 32) * 32 * t16_prof_words(R, DNA, sc.A) * sizeof(uint32_t);
}

// resident blocks per SM of one variant (0 when it cannot launch)
template <int R, bool DNA>
int t16_blocks(const Scoring &sc) {
    const size_t smem = t16_smem_bytes<R, DNA>(sc);
    if (cudaFuncSetAttribute(k_trace16<R, DNA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace16<R, DNA>, kT16Block, smem) != cudaSuccess)
        return 0;
    return n;
}

template <int R, bool DNA>
cudaError_t t16_launch(const BatchView &b, const Scoring &sc, const T16Scratch &ts, int sms, int cls,
                       cudaStream_t st) {
    const int v = cls - kTraceT16First;
    if (ts.dir_words[v] <= 0 || ts.warps[v] <= 0) return cudaSuccess;  // no pairs of the class
    const int per_sm = t16_blocks<R, DNA>(sc);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(sms * per_sm, ts.warps[v] / (kT16Block / 32)));
    k_trace16<R, DNA><<<grid, kT16Block, t16_smem_bytes<R, DNA>(sc), st>>>(b, sc, ts, cls);
    return cudaGetLastError();
}

}  // namespace

int t16_max_warps(const Scoring &sc, int sms, int v) {
    int per_sm = 0;
    if (sc.dna4) {
        switch (v) {
        case 0: per_sm = t16_blocks<4, true>(sc); break;
        case 1: per_sm = t16_blocks<8, true>(sc); break;
        case 2: per_sm = t16_blocks<12, true>(sc); break;
        default: per_sm = t16_blocks<16, true>(sc); break;
        }
    } else if (v <= 1) {
        per_sm = v == 0 ? t16_blocks<4, false>(sc) : t16_blocks<8, false>(sc);
    }
    return std::max(0, sms * per_sm) * (kT16Block / 32);
}

cudaError_t launch_trace16(const BatchView &b, const Scoring &sc, const T16Scratch &ts, int sms, cudaStream_t st) {
    cudaError_t e;
    const int c0 = kTraceT16First;
    if (sc.dna4) {
        if ((e = t16_launch<16, true>(b, sc, ts, sms, c0 + 3, st))) return e;
        if ((e = t16_launch<12, true>(b, sc, ts, sms, c0 + 2, st))) return e;
        if ((e = t16_launch<8, true>(b, sc, ts, sms, c0 + 1, st))) return e;
        if ((e = t16_launch<4, true>(b, sc, ts, sms, c0, st))) return e;
    } else {
        if ((e = t16_launch<8, false>(b, sc, ts, sms, c0 + 1, st))) return e;
        if ((e = t16_launch<4, false>(b, sc, ts, sms, c0, st))) return e;
    }
    return cudaSuccess;
}

}  // namespace gsw
