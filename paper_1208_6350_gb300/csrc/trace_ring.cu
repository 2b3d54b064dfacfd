// Banded global Gotoh with the traceback that emits the CIGAR, for bands too
// wide for the anti-diagonal warp kernels ("Algorithm and implementation",
// item (1): the detailed alignment comes from a banded SW between the begin
// and the end).
//
// Region.  Rows i in [1, la] (query), columns j in [1, lb] (target), row and
// column 0 the global boundary.  The provable band is the diagonals
// dlo <= j - i <= dhi (band_range).  Strip x holds rows
// [1 + 512x, 512(x+1)] and the columns [c0(x), c1(x)] that the band reaches
// in those rows, so the region computed is a staircase that contains the
// band.  Any region between the band and the full rectangle gives the
// canonical traceback: an optimal path lies in the band, so its cells keep
// their full-rectangle values, and a predecessor that ties on the full
// rectangle is itself on an optimal path; cells outside the region are -inf.
//
// Fill.  One warp per strip, 32 lanes x 16 rows, 32-bit lanes, one target
// column per lane and step as in the local fill (lane k at step s works on
// column c0 + s - k, receives H and F of the row above from lane k-1 by
// shuffle; lane 0 reads the previous strip's bottom row from global memory,
// one block of 32 columns ahead).  The strips of a pair run on the warps of a
// CTA in phases separated by a barrier, each strip far enough behind the one
// above (ring_lag) that every boundary word it reads was written in a
// completed phase; several pairs are in flight per CTA.  Per cell 4 bits go
// to global memory: H differs from the diagonal term (bit 0), H differs from E
// (bit 1), E extends rather than opens here (bit 2), F extends rather than
// opens here (bit 3); lane k's 16 rows of one step form two words (rows 0-7,
// rows 8-15), so a warp writes 256 contiguous bytes per step.
//
// Walk.  One warp per pair stages tiles of 32 steps x 32 lanes x 2 direction
// words in shared memory and lane 0 walks from (la, lb) in state H with the
// fixed preference (diagonal, then E, then F; open before extend), emitting
// runs (len << 4) | op in reverse, then the warp writes them forward.  While
// lane 0 walks one tile the other lanes copy the 32 steps below it (where the
// path goes next unless it leaves the strip) into a second buffer.
#include "gsw_impl.cuh"

#include <climits>

namespace gsw {

int ring_trace_class() { return 4; }

namespace {

constexpr int kRP = 32;          // lanes per strip
constexpr int kRR = 16;          // rows per lane
constexpr int kRS = kRP * kRR;   // rows per strip
constexpr int kRWords = kRR / 8; // direction words per lane and step (8 rows of 4 bits each)
constexpr int kRStep = kRP * kRWords;  // direction words of one step of a strip
constexpr int kRW = 8;           // warps per CTA
constexpr int kRC = 64;          // steps per phase
constexpr int kRSlots = 4;       // pairs in flight per CTA
constexpr int kRNeg = -(1 << 28);
constexpr int kRTile = 32;       // steps of direction words in each of the walk's two tiles

// Geometry of one pair's banded DP.
struct RingGeom {
    int la, lb, dlo, dhi, nstrips, stride;
    __device__ int c0(int x) const { return max(1, 1 + x * kRS + dlo); }
    __device__ int c1(int x) const { return min(lb, min((x + 1) * kRS, la) + dhi); }
    __device__ long long words() const { return (long long)nstrips * stride * kRStep; }
};

__device__ __forceinline__ bool ring_geom(const gsw_result &r, const Scoring &sc, RingGeom *g) {
    g->la = r.read_end1 - r.read_begin1 + 1;
    g->lb = r.ref_end1 - r.ref_begin1 + 1;
    int dlo, dhi;
    band_range(g->la, g->lb, r.score1, sc, &dlo, &dhi);
    g->dlo = dlo;
    g->dhi = dhi;
    g->nstrips = (g->la + kRS - 1) / kRS;
    // steps of the widest strip: its columns plus the 31-step wavefront skew
    g->stride = min(g->lb, kRS + dhi - dlo) + kRP;
    return g->la >= 1 && g->lb >= 1 && dlo <= 0 && dhi >= g->lb - g->la;
}

// Phases strip x+1 trails strip x: strip x writes column j at its step
// j - c0(x) + 31, strip x+1 reads columns up to c0(x+1) + s + 63 at its step
// s, and c0(x+1) - c0(x) <= 512, so (lag - 1) * 64 >= 512 + 63 + 31.
constexpr int kRingLag = 1 + (kRS + 2 * kRP - 1 + kRP - 1 + kRC - 1) / kRC;

// Profile index of (letter a, row r, lane l): lane-minor groups of 4 rows.
__device__ __forceinline__ int ridx(int a, int r, int l) { return ((a * (kRR / 4) + r / 4) * 32 + l) * 4 + (r & 3); }

struct RingJob {
    const uint8_t *q, *t;  // q[i - 1], t[j - 1] for grid row i, column j
    RingGeom g;
    uint32_t *dirs;        // nstrips x stride x 32 words
    int2 *bnd;             // 2 x lb boundary words (H, F of a strip's bottom row)
    int *final_h;          // H(la, lb)
};

// bits |= m when a != b: a compare into a predicate and a predicated or
__device__ __forceinline__ void or_if_ne(uint32_t &bits, int a, int b, uint32_t m) {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(bits)
        : "r"(a), "r"(b), "r"(m));
}

// One strip of the banded fill for lane k of a warp.
struct BandStrip {
    RingJob job;
    const int8_t *W;
    int A, O, X;
    uint32_t *psm;
    int k, x, c0, c1, c1a, nsteps, i0;
    int fin_j;     // column of H(la, lb) when one of this lane's rows is la, else -1
    bool first, last, bo;  // bo: this lane writes the strip's bottom row
    const int2 *bin;
    int2 *bout;
    uint32_t *dout;
    int HO[kRR], E[kRR];  // H(i, j) - O and E(i, j + 1) of the lane's rows
    int hdiag, xh, xf;     // H values are all kept as H - O
    int2 b_cur, b_nxt;  // boundary words of the current and next 32 columns
    int l_cur, l_nxt;   // target letters of the same columns
    int a_prev;         // target letter this lane used at the previous step

    __device__ void begin(const RingJob &jb, const Scoring &sc, const int8_t *sW, uint32_t *psm_, int lane, int x_) {
        job = jb;
        W = sW;
        A = sc.A;
        O = sc.O;
        X = sc.X;
        psm = psm_;
        k = lane;
        x = x_;
        const RingGeom &g = job.g;
        c0 = g.c0(x);
        c1 = g.c1(x);
        c1a = x > 0 ? g.c1(x - 1) : 0;
        nsteps = c1 - c0 + 1 + kRP - 1;
        i0 = 1 + x * kRS + k * kRR;
        first = x == 0;
        last = x == g.nstrips - 1;
        bo = k == kRP - 1 && !last;
        fin_j = (i0 <= g.la && g.la < i0 + kRR) ? g.lb : -1;
        // boundary word of column j at [j - 1]
        bin = job.bnd + (size_t)((x + 1) & 1) * g.lb;
        bout = job.bnd + (size_t)(x & 1) * g.lb;
        dout = job.dirs + (size_t)x * g.stride * kRStep;
        // profile: W(q_i, a) + O of this lane's rows (W = 0 below the last
        // row); with H kept as H - O the diagonal term is one add
        for (int r = 0; r < kRR; r++) {
            const int i = i0 + r;
            const int qa = i <= g.la ? min((int)job.q[i - 1], A - 1) : -1;
            for (int a = 0; a < A; a++) psm[ridx(a, r, k)] = (uint32_t)((qa >= 0 ? (int)W[qa * A + a] : 0) + O);
        }
        __syncwarp();
        // left boundary: column c0 - 1 is column 0 (H = -O - (i-1)X) or outside (-inf)
#pragma unroll
        for (int r = 0; r < kRR; r++) {
            HO[r] = (c0 == 1 ? -O - (i0 + r - 1) * X : kRNeg) - O;
            E[r] = c0 == 1 ? HO[r] : kRNeg;  // E(i, c0) = H(i, 0) - O
        }
        // H(i0 - 1, c0 - 1), the first diagonal input of lane 0
        const int ia = i0 - 1, ja = c0 - 1;
        if (ja == 0) hdiag = (ia == 0 ? 0 : -O - (ia - 1) * X) - O;
        else if (first) hdiag = -O - (ja - 1) * X - O;
        else hdiag = ja <= c1a ? bin[ja - 1].x : kRNeg - O;
        // H of the row above this lane's first row, at column c0 - 1: lane k
        // takes it as the diagonal input of its first column
        xh = (c0 == 1 ? (i0 == 1 ? 0 : -O - (i0 - 2) * X) : kRNeg) - O;
        xf = kRNeg;
        b_cur = make_int2(kRNeg - O, kRNeg);
        b_nxt = b_cur;
        l_cur = l_nxt = a_prev = 0;
        prefetch(0);
    }

    // lane k loads the boundary word (H - O, F of the row below) of column
    // c0 + s0 + k (columns the strip above did not reach are -inf) and the
    // target letter of that column (lane 0 takes it at step s0 + k; the other
    // lanes get their letters from the lane before, one step later)
    __device__ __forceinline__ void prefetch(int s0) {
        const int j = c0 + s0 + k;
        b_nxt = (j <= c1a) ? bin[j - 1] : make_int2(kRNeg - O, kRNeg);
        l_nxt = j <= c1 ? min((int)job.t[j - 1], A - 1) : 0;
    }

    __device__ __forceinline__ void step(int s, uint32_t *dp) {
        const int j = c0 + s - k;
        const int bi = s & (kRP - 1);
        if (bi == 0) {
            b_cur = b_nxt;
            l_cur = l_nxt;
            prefetch(s + kRP);
        }
        int a = __shfl_up_sync(0xFFFFFFFFu, a_prev, 1);
        const int a0 = __shfl_sync(0xFFFFFFFFu, l_cur, bi);
        int hin = xh, fin = xf;
        if (first) {
            if (k == 0) {
                hin = -O - (j - 1) * X - O;  // H(0, j) - O
                fin = hin;                   // F(1, j) = H(0, j) - O: F(0, j) = -inf
            }
        } else {
            const int hb = __shfl_sync(0xFFFFFFFFu, b_cur.x, bi);
            const int fb = __shfl_sync(0xFFFFFFFFu, b_cur.y, bi);
            if (k == 0) {
                hin = hb;
                fin = fb;
            }
        }
        if (k == 0) a = a0;
        a_prev = a;
        int diag = hdiag;
        hdiag = hin;
        int houp = hin, f = fin;
        uint32_t bits[kRWords] = {};
        if ((unsigned)(j - c0) <= (unsigned)(c1 - c0)) {
            int w[kRR];
#pragma unroll
            for (int r = 0; r < kRR; r += 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(psm + ridx(a, r, k));
                w[r] = (int)v.x; w[r + 1] = (int)v.y; w[r + 2] = (int)v.z; w[r + 3] = (int)v.w;
            }
#pragma unroll
            for (int r = 0; r < kRR; r++) {
                const int holeft = HO[r];  // H(i, j-1) - O: where E(i, j) opens
                const int e = E[r];
                const int dw = diag + w[r];  // H(i-1, j-1) + W(q_i, t_j)
                const int h = __vimax3_s32(dw, e, f);  // three-input max, one instruction
                // one compare and one predicated or per bit
                uint32_t &bw = bits[r / 8];
                const int sh = 4 * (r % 8);
                or_if_ne(bw, h, dw, 1u << sh);      // H not from the diagonal
                or_if_ne(bw, h, e, 2u << sh);       // H not from E
                or_if_ne(bw, e, holeft, 4u << sh);  // E(i, j) extends, not opened
                or_if_ne(bw, f, houp, 8u << sh);    // F(i, j) extends, not opened
                const int ho = h - O;
                E[r] = __viaddmax_s32(e, -X, ho);  // max(e - X, ho), one instruction
                f = __viaddmax_s32(f, -X, ho);
                diag = holeft;
                houp = ho;
                HO[r] = ho;
            }
            if (j == fin_j) {
#pragma unroll
                for (int r = 0; r < kRR; r++)
                    if (i0 + r == job.g.la) *job.final_h = HO[r] + O;
            }
            if (bo) bout[j - 1] = make_int2(HO[kRR - 1], f);
        }
        static_assert(kRWords == 2, "one 8-byte store per lane and step");
        *reinterpret_cast<uint2 *>(dp) = make_uint2(bits[0], bits[1]);
        xh = __shfl_up_sync(0xFFFFFFFFu, HO[kRR - 1], 1);
        xf = __shfl_up_sync(0xFFFFFFFFu, f, 1);
    }

    // steps [s0, s1); true when the strip is complete
    __device__ bool run(int s0, int s1) {
        s1 = min(s1, nsteps);
        uint32_t *dp = dout + (size_t)s0 * kRStep + k * kRWords;
#pragma unroll 1
        for (int s = s0; s < s1; s++, dp += kRStep) step(s, dp);
        return s1 >= nsteps;
    }
};

struct RingSlot {
    RingJob job;
    int pair;        // -1: free
    int seq;
    int next;        // next strip to hand out
    int last_start;  // phase the last handed-out strip started
    int running;
};

struct RingCmd {
    int slot, strip, start;
};

struct RingShared {
    RingSlot slot[kRSlots];
    RingCmd cmd[kRW];
    int ended[kRW];
    int seq, exhausted, done;
};
// (kRW warps per CTA, or kRW / 2 when a large alphabet's profiles would not
// fit the shared memory of 8 warps)

// Pairs of the ring class in plan order: t in [g0, g1) of the group; the
// pair's direction words start at prefix[t] - prefix[g0] in the pool.
struct RingLaunch {
    BatchView b;
    Scoring sc;
    const int32_t *order;     // sorted pair indices (the class starts at var_start[cls])
    const int32_t *var_start;
    int cls;
    const long long *prefix;  // [n + 1] direction words before each pair of the class
    int *final_h;             // [n]
    int *group;               // [0] g0, [1] g1, [2] head
    uint32_t *pool;
    long long pool_words;
    int2 *bnd;                // per slot 2 x ncap
    long long bnd_stride;     // int2 per slot
    uint32_t *ops;            // walk: per warp op_words
    long long op_words;
};

__device__ bool ring_open(const RingLaunch &rl, RingSlot &S, int s, int seq) {
    const int g0 = rl.group[0], g1 = rl.group[1];
    const int t = g0 + atomicAdd(&rl.group[2], 1);
    if (t >= g1) return false;
    const int pair = rl.order[rl.var_start[rl.cls] + t];
    const gsw_result r = rl.b.res[pair];
    RingJob jb;
    if (!ring_geom(r, rl.sc, &jb.g) || jb.g.words() > rl.pool_words || 2LL * jb.g.lb > rl.bnd_stride) {
        rl.b.res[pair].flags |= kResInternal;
        rl.final_h[t] = INT_MIN;
        S.pair = -1;
        return true;  // taken (and rejected); try the next one
    }
    jb.q = rl.b.q + rl.b.q_off[pair] + r.read_begin1;
    jb.t = rl.b.t + rl.b.t_off[pair] + r.ref_begin1;
    jb.dirs = rl.pool + (rl.prefix[t] - rl.prefix[g0]);
    jb.bnd = rl.bnd + (size_t)(blockIdx.x * kRSlots + s) * rl.bnd_stride;
    jb.final_h = rl.final_h + t;
    rl.final_h[t] = INT_MIN;
    S.job = jb;
    S.pair = pair;
    S.seq = seq;
    S.next = 0;
    S.last_start = 0;
    S.running = 0;
    return true;
}

__device__ void ring_schedule(const RingLaunch &rl, RingShared &sh, int ph, int nw) {
    for (int w = 0; w < nw; w++) {
        if (!sh.ended[w]) continue;
        sh.ended[w] = 0;
        RingSlot &S = sh.slot[sh.cmd[w].slot];
        S.running--;
        if (S.running == 0 && S.next == S.job.g.nstrips) S.pair = -1;
        sh.cmd[w].slot = -1;
    }
    for (int w = 0; w < nw; w++) {
        RingCmd &c = sh.cmd[w];
        if (c.slot >= 0) continue;
        int pick = -1, best = INT_MAX;
        for (int s = 0; s < kRSlots; s++) {
            const RingSlot &S = sh.slot[s];
            if (S.pair >= 0 && S.next < S.job.g.nstrips && (S.next == 0 || ph >= S.last_start + kRingLag) &&
                S.seq < best) {
                best = S.seq;
                pick = s;
            }
        }
        while (pick < 0 && !sh.exhausted) {
            int fs = -1;
            for (int s = 0; s < kRSlots; s++)
                if (sh.slot[s].pair < 0) { fs = s; break; }
            if (fs < 0) break;
            if (!ring_open(rl, sh.slot[fs], fs, sh.seq)) {
                sh.exhausted = 1;
                break;
            }
            if (sh.slot[fs].pair >= 0) {
                sh.seq++;
                pick = fs;
            }
        }
        if (pick < 0) break;
        RingSlot &S = sh.slot[pick];
        c.slot = pick;
        c.strip = S.next++;
        c.start = ph;
        S.last_start = ph;
        S.running++;
    }
    bool busy = !sh.exhausted;
    for (int s = 0; s < kRSlots; s++) busy |= sh.slot[s].pair >= 0;
    sh.done = busy ? 0 : 1;
}

template <bool DNA>
__global__ void __launch_bounds__(kRW * 32, 1) k_trace_ring(RingLaunch rl) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ RingShared sh;
    __shared__ int8_t sW[kMaxAlpha * kMaxAlpha];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int A = DNA ? 4 : rl.sc.A;
    for (int i = threadIdx.x; i < rl.sc.A * rl.sc.A; i += blockDim.x) sW[i] = rl.sc.W[i];
    uint32_t *psm = smem + (size_t)warp * A * kRR * 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRSlots; s++) sh.slot[s].pair = -1;
        for (int w = 0; w < kRW; w++) {
            sh.cmd[w].slot = -1;
            sh.ended[w] = 0;
        }
        sh.seq = 0;
        sh.exhausted = 0;
        sh.done = 0;
    }
    BandStrip bs;
#pragma unroll 1
    for (int ph = 0;; ph++) {
        __syncthreads();
        if (threadIdx.x == 0) ring_schedule(rl, sh, ph, nw);
        __syncthreads();
        if (sh.done) break;
        const RingCmd cmd = sh.cmd[warp];
        if (cmd.slot < 0) continue;
        if (ph == cmd.start) bs.begin(sh.slot[cmd.slot].job, rl.sc, sW, psm, lane, cmd.strip);
        const int q = ph - cmd.start;
        if (bs.run(q * kRC, (q + 1) * kRC) && lane == 0) sh.ended[warp] = 1;
    }
}

// Group t in [g0, g1): the pairs whose direction words fit the pool.
__global__ void k_ring_group(const long long *prefix, const int32_t *var_start, int cls, long long pool_words,
                             int *group) {
    const int n = var_start[cls + 1] - var_start[cls];
    const int g0 = group[0];
    int lo = g0, hi = n;  // largest g1 with prefix[g1] - prefix[g0] <= pool
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] - prefix[g0] <= pool_words) lo = mid;
        else hi = mid - 1;
    }
    group[1] = (lo == g0 && g0 < n) ? g0 + 1 : lo;  // a pair beyond the pool is rejected alone
    group[2] = 0;
}

__global__ void k_ring_advance(int *group) { group[0] = group[1]; }

// Direction words (and walk op words) of each pair of the class, then the
// exclusive prefix over the class in plan order (one block).
__global__ void __launch_bounds__(1024) k_ring_needs(BatchView b, Scoring sc, const int32_t *order,
                                                     const int32_t *var_start, int cls, long long *prefix,
                                                     unsigned long long *out) {
    const int cls_start = var_start[cls], n = var_start[cls + 1] - cls_start;
    __shared__ long long part[1024];
    __shared__ long long carry;
    __shared__ unsigned long long mx_words, mx_ops;
    if (threadIdx.x == 0) {
        carry = 0;
        mx_words = 0;
        mx_ops = 0;
    }
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int t = base + threadIdx.x;
        long long w = 0;
        if (t < n) {
            const gsw_result r = b.res[order[cls_start + t]];
            RingGeom g;
            if (ring_geom(r, sc, &g)) {
                w = g.words();
                atomicMax(&mx_words, (unsigned long long)w);
                atomicMax(&mx_ops, (unsigned long long)(g.la + g.lb + 2));
            }
        }
        part[threadIdx.x] = w;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {
            const long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (t < n) prefix[t] = carry + part[threadIdx.x] - w;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[n] = carry;
        out[0] = (unsigned long long)carry;
        out[1] = mx_words;
        out[2] = mx_ops;
    }
}

// Walk of one pair by one warp (see the file comment).
// A warp copies `steps` steps of direction words (kRStep words, 256 bytes
// each, 16-byte aligned: every pair's words start at a multiple of kRStep
// words) into shared memory without waiting; walk_copy_wait waits for this
// lane's copies.
__device__ __forceinline__ void walk_copy(uint32_t *dst, const uint32_t *src, int steps, int lane) {
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(dst);
    for (int c = lane; c < steps * (kRStep / 4); c += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16u * c), "l"(src + 4 * c) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void walk_copy_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kWalkWarps = 2;  // warps per block: two 16 KB tile pairs

__global__ void __launch_bounds__(kWalkWarps * 32) k_ring_walk(RingLaunch rl) {
    __shared__ __align__(16) uint32_t tile[kWalkWarps][2][kRTile * kRStep];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * kWalkWarps + warp, nwarps = gridDim.x * kWalkWarps;
    uint32_t (*stage)[kRTile * kRStep] = tile[warp];
    uint32_t *ops = rl.ops + (size_t)gwarp * rl.op_words;
    const int g0 = rl.group[0], g1 = rl.group[1];
    for (int t = g0 + gwarp; t < g1; t += nwarps) {
        const int pair = rl.order[rl.var_start[rl.cls] + t];
        gsw_result *rp = rl.b.res + pair;
        const gsw_result r = *rp;
        RingGeom g;
        bool ok = ring_geom(r, rl.sc, &g) && rl.final_h[t] == r.score1 && g.la + g.lb + 2 <= rl.op_words;
        if (!ok) {
            if (lane == 0 && !(r.flags & kResInternal)) rp->flags |= kResInternal;
            continue;
        }
        const uint32_t *dirs = rl.pool + (rl.prefix[t] - rl.prefix[g0]);
        int i = g.la, j = g.lb, st = 0, cur = -1, len = 0, runs = 0;
        // staged tiles: strip and step range [lo, hi] of the current buffer
        // and of the one being filled ahead of it (the steps just below, in
        // the same strip, where the walk goes next unless it leaves the strip)
        int cx = -1, clo = 0, chi = -1, px = -1, plo = 0, phi = -1, buf = 0;
        while (ok && i > 0 && j > 0) {
            const int x = (i - 1) / kRS;
            const int k = ((i - 1) % kRS) / kRR;
            const int c0 = g.c0(x);
            if (j < c0 || j > g.c1(x)) {  // left the region (never for an optimal path)
                ok = false;
                break;
            }
            const int s = j - c0 + k;
            if (x != cx || s < clo || s > chi) {
                walk_copy_wait();
                __syncwarp();
                if (x == px && s >= plo && s <= phi) {
                    buf ^= 1;
                    cx = px, clo = plo, chi = phi;
                } else {
                    cx = x, chi = s, clo = max(0, s - kRTile + 1);
                    walk_copy(stage[buf], dirs + ((size_t)x * g.stride + clo) * kRStep, chi - clo + 1, lane);
                    walk_copy_wait();
                    __syncwarp();
                }
                px = -1;
                if (clo > 0) {
                    px = cx, phi = clo - 1, plo = max(0, clo - kRTile);
                    walk_copy(stage[buf ^ 1], dirs + ((size_t)px * g.stride + plo) * kRStep, phi - plo + 1, lane);
                }
            }
            if (lane == 0) {
                // walk inside the tile: idx = (s - clo) * kRStep + 2k + r / 8,
                // the word of row i (lane k, row r of the lane) at column j;
                // d = j - c0 (the region's left edge)
                const uint32_t *tl = stage[buf];
                int kk = k, r = (i - 1) % kRR, sh = 4 * (r % 8), d = j - c0;
                int idx = (s - clo) * kRStep + kRWords * k + r / 8;
                while (i > 0 && j > 0 && idx >= 0 && kk >= 0) {
                    if (d < 0) {  // left the region
                        ok = false;
                        break;
                    }
                    const uint32_t wd = tl[idx] >> sh;
                    int op;
                    bool up, left;
                    if (st == 0 && !(wd & 1)) {
                        op = GSW_CIGAR_M;  // preference: the diagonal, then E, then F
                        up = left = true;
                    } else {
                        if (st == 0) st = (wd & 2) ? 2 : 1;
                        if (st == 1) {
                            op = GSW_CIGAR_D;
                            st = (wd & 4) ? 1 : 0;
                            up = false;
                            left = true;
                        } else {
                            op = GSW_CIGAR_I;
                            st = (wd & 8) ? 2 : 0;
                            up = true;
                            left = false;
                        }
                    }
                    if (left) {
                        j--;
                        d--;
                        idx -= kRStep;
                    }
                    if (up) {
                        i--;
                        if (--r < 0) {  // the lane above, one step earlier: its row 15
                            r = kRR - 1;
                            kk--;
                            idx -= kRStep + 1;
                            sh = 28;
                        } else if (r == 7) {  // row 7: the lane's first word
                            idx -= 1;
                            sh = 28;
                        } else {
                            sh -= 4;
                        }
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
        }
        walk_copy_wait();
        __syncwarp();
        if (lane == 0 && ok) {
            // row 0 or column 0: the rest is one gap (D along row 0, I along column 0)
            const int rest_op = i == 0 ? GSW_CIGAR_D : GSW_CIGAR_I;
            const int rest = i == 0 ? j : i;
            if (rest > 0) {
                if (rest_op == cur) {
                    len += rest;
                } else {
                    if (len) ops[runs++] = ((uint32_t)len << 4) | (uint32_t)cur;
                    cur = rest_op;
                    len = rest;
                }
            }
            if (len) ops[runs++] = ((uint32_t)len << 4) | (uint32_t)cur;
        }
        const int nr = __shfl_sync(0xFFFFFFFFu, runs, 0);
        if (!ok) {
            if (lane == 0) rp->flags |= kResInternal;
            __syncwarp();
            continue;
        }
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(rl.b.cigar_cursor, (unsigned long long)nr);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if ((long long)(off + nr) > rl.b.cigar_cap) {
            if (lane == 0) {
                rp->flags |= GSW_RES_CIGAR_SPACE;
                rp->cigar_len = -nr;
                rp->cigar_off = -1;
                rp->flags &= ~kResPendingTrace;
            }
            __syncwarp();
            continue;
        }
        __syncwarp();
        for (int q = lane; q < nr; q += 32) rl.b.cigar[off + q] = ops[nr - 1 - q];
        if (lane == 0) {
            rp->cigar_len = nr;
            rp->cigar_off = (int64_t)off;
            rp->flags &= ~kResPendingTrace;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_ring_needs(const BatchView &b, const Scoring &sc, const int32_t *order, const int32_t *var_start,
                              long long *prefix, unsigned long long *out, cudaStream_t st) {
    k_ring_needs<<<1, 1024, 0, st>>>(b, sc, order, var_start, ring_trace_class(), prefix, out);
    return cudaGetLastError();
}

// One group: bounds, banded fill, walk, advance.  `rl` holds the pool, the
// slot boundary buffers and the walk's op buffers.
cudaError_t launch_ring_group(const RingLaunchArgs &a, int sms, cudaStream_t st) {
    RingLaunch rl;
    rl.b = a.b;
    rl.sc = a.sc;
    rl.order = a.order;
    rl.var_start = a.var_start;
    rl.cls = ring_trace_class();
    rl.prefix = a.prefix;
    rl.final_h = a.final_h;
    rl.group = a.group;
    rl.pool = a.pool;
    rl.pool_words = a.pool_words;
    rl.bnd = a.bnd;
    rl.bnd_stride = a.bnd_stride;
    rl.ops = a.ops;
    rl.op_words = a.op_words;
    k_ring_group<<<1, 1, 0, st>>>(a.prefix, a.var_start, rl.cls, a.pool_words, a.group);
    const bool dna = a.sc.dna4 != 0;
    const int A = dna ? 4 : a.sc.A;
    const size_t per_warp = (size_t)A * kRR * 32 * sizeof(uint32_t);
    const int nw = per_warp * kRW <= 200 * 1024 ? kRW : kRW / 2;
    const size_t smem = per_warp * nw;
    int nb = 0;
    if (dna) {
        cudaFuncSetAttribute(k_trace_ring<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace_ring<true>, nw * 32, smem);
    } else {
        cudaFuncSetAttribute(k_trace_ring<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace_ring<false>, nw * 32, smem);
    }
    if (nb < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(sms * nb, a.slots / kRSlots);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (dna) k_trace_ring<true><<<grid, nw * 32, smem, st>>>(rl);
    else k_trace_ring<false><<<grid, nw * 32, smem, st>>>(rl);
    const int wgrid = std::max(1, a.walk_warps / kWalkWarps);
    k_ring_walk<<<wgrid, kWalkWarps * 32, 0, st>>>(rl);
    k_ring_advance<<<1, 1, 0, st>>>(a.group);
    return cudaGetLastError();
}

int ring_slots_per_cta() { return kRSlots; }

}  // namespace gsw
