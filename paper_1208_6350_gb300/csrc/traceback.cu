// Banded global Gotoh between begin and end, with the traceback that emits the
// CIGAR on the device ("Algorithm and implementation", item (1): the banded SW
// whose band is defined by the beginning and ending positions generates the
// detailed alignment).
//
// The band is the provable one (band_halfwidth): every diagonal that can
// carry a path scoring score1.  Inside it, every cell of every optimal path
// has the value of the full-rectangle DP, so each traceback comparison decides
// exactly as on the full rectangle and the CIGAR is the canonical one.
//
// One warp per pair.  Lanes hold consecutive diagonals (chunks of 32); rows
// are processed top to bottom.  F comes from the row above (diagonal + 1, a
// shuffle), the diagonal term from the same lane; E, the left-to-right gap
// state, is a prefix maximum over the row: E(i,j) = max_{k<j}(H(i,k) + kX) -
// O - (j-1)X, and since O >= X it may be taken over H without E (H0), so one
// warp scan per chunk gives it.  Each cell's 4 decision bits (H source:
// diagonal / E / F; E opened here; F opened here) are stored as 4 ballot bit
// planes per row and chunk.  Lane 0 then walks back from (la, lb).
#include "gsw_impl.cuh"

#include <climits>

namespace gsw {
namespace {

constexpr int kTBlock = 128;
constexpr int kAdwMaxChunks = 256;  // widest band of the wide anti-diagonal kernel: 64 x 256 diagonals
constexpr int kNegT = -(1 << 28);
constexpr int kNegHalf = -(1 << 27);

struct TraceCfg {
    int smem_dir_words;  // per warp, shared memory
    int smem_op_words;
    int smem_state_chunks;
};

__device__ __forceinline__ int sw(const Scoring &sc, int a, int b) { return sc.W[a * sc.A + b]; }

// Needs of one pair, in words: direction planes, reversed ops, chunk state.
struct Need {
    long long dir, ops;
    int nch, dlo, dhi;
};

__device__ Need pair_need(const gsw_result &r, const Scoring &sc) {
    Need nd{0, 0, 0, 0, 0};
    const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
    int dlo, dhi;
    const int width = band_range(la, lb, r.score1, sc, &dlo, &dhi);
    nd.dlo = dlo;
    nd.dhi = dhi;
    nd.nch = 0;
    if (width <= 512) {
        // anti-diagonal kernel: (la + lb + 1) steps x chunks of 64 x 4 planes
        const int nch_cls = width <= 64 ? 1 : width <= 128 ? 2 : width <= 256 ? 4 : 8;
        nd.dir = (long long)(la + lb + 1) * nch_cls * 4;
        nd.ops = (long long)la + lb + 2;
    } else if (width <= 64 * kAdwMaxChunks) {
        nd.nch = (width + 63) / 64;  // wide anti-diagonal kernel
        nd.dir = (long long)(la + lb + 1) * nd.nch * 4;
        nd.ops = (long long)la + lb + 2;
    } else {
        nd.nch = -((dhi - dlo + 32) / 32);  // row kernel (negative: marks the class)
        nd.dir = (long long)(la + 1) * (-nd.nch) * 4;
        nd.ops = (long long)la + lb + 2;
    }
    return nd;
}

__device__ __forceinline__ int dhi_width_chunks(const Need &nd) { return (nd.dhi - nd.dlo + 32) / 32; }

// pairs the thread-per-pair band kernel left to this kernel (band too wide)
__device__ __forceinline__ bool wants_trace(const gsw_result &r) {
    return r.score1 > 0 && (r.flags & kResPendingTrace) && !(r.flags & kResInternal) && r.read_begin1 >= 0 &&
           r.ref_begin1 >= 0;
}

__global__ void k_trace_need(BatchView b, Scoring sc, unsigned long long *max_need) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (p < b.npairs) {
        const gsw_result r = b.res[p];
        const Need nd = wants_trace(r) ? pair_need(r, sc) : Need{0, 0, 1, 0, 0};
        if (nd.nch == 0) {  // at most 512 diagonals (wider bands: trace_ring.cu)
            const int g = 0;
            v[g] = (unsigned)min(nd.dir, (long long)UINT_MAX);
            v[g + 1] = (unsigned)min(nd.ops, (long long)UINT_MAX);
            v[g + 2] = (unsigned)(nd.nch < 0 ? -nd.nch : (nd.nch > 0 ? nd.nch : 1));
        }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const unsigned m = __reduce_max_sync(0xFFFFFFFFu, v[k]);
        if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&max_need[k], (unsigned long long)m);
    }
}

__device__ void trace_pair(const BatchView &b, const Scoring &sc, int p, const gsw_result &r, const Need &nd,
                           uint32_t *dirs, uint32_t *ops, int *stH, int *stF, int lane) {
    const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
    const uint8_t *qs = b.q + b.q_off[p] + r.read_begin1;
    const uint8_t *ts = b.t + b.t_off[p] + r.ref_begin1;
    const int O = sc.O, X = sc.X;
    const int nch = nd.nch, dlo = nd.dlo, dhi = nd.dhi;
    for (int c = 0; c < nch; c++) {
        stH[c * 32 + lane] = kNegT;
        stF[c * 32 + lane] = kNegT;
    }
    __syncwarp();
    int final_h = kNegT;
    for (int i = 0; i <= la; i++) {
        int carry_a = kNegT, carry_h = kNegT;
        const int qa = i >= 1 ? min((int)qs[i - 1], sc.A - 1) : 0;
        for (int c = 0; c < nch; c++) {
            const int d = dlo + 32 * c + lane;
            const int j = i + d;
            const bool valid = d <= dhi && j >= 0 && j <= lb;
            const int hp = stH[c * 32 + lane], fp = stF[c * 32 + lane];
            int hup = __shfl_down_sync(0xFFFFFFFFu, hp, 1);
            int fup = __shfl_down_sync(0xFFFFFFFFu, fp, 1);
            if (lane == 31) {
                hup = c + 1 < nch ? stH[(c + 1) * 32] : kNegT;
                fup = c + 1 < nch ? stF[(c + 1) * 32] : kNegT;
            }
            int F = kNegT, hdg = kNegT, H0;
            bool fopen = false;
            if (i == 0) {
                H0 = j == 0 ? 0 : kNegT;
            } else {
                const int fo = hup - O, fe = fup - X;
                F = max(fo, fe);
                fopen = F == fo;
                if (j >= 1 && valid) hdg = hp + sw(sc, qa, min((int)ts[j - 1], sc.A - 1));
                H0 = max(hdg, F);
            }
            if (!valid || H0 < kNegHalf) { H0 = kNegT; }
            if (!valid || F < kNegHalf) F = kNegT;
            const int A = H0 > kNegHalf ? H0 + j * X : kNegT;
            int incl = A;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl = max(incl, v);
            }
            int excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
            excl = lane == 0 ? carry_a : max(excl, carry_a);
            carry_a = max(carry_a, __shfl_sync(0xFFFFFFFFu, incl, 31));
            int E = excl > kNegHalf ? excl - O - (j - 1) * X : kNegT;
            int H = max(H0, E);
            if (!valid) { H = kNegT; E = kNegT; }
            const int src = (i >= 1 && j >= 1 && H == hdg && hdg > kNegHalf) ? 0 : (H == E ? 1 : 2);
            int hleft = __shfl_up_sync(0xFFFFFFFFu, H, 1);
            if (lane == 0) hleft = carry_h;
            carry_h = __shfl_sync(0xFFFFFFFFu, H, 31);
            const bool eopen = E > kNegHalf && E == hleft - O;
            __syncwarp();
            stH[c * 32 + lane] = H;
            stF[c * 32 + lane] = F;
            const unsigned b0 = __ballot_sync(0xFFFFFFFFu, src & 1);
            const unsigned b1 = __ballot_sync(0xFFFFFFFFu, src & 2);
            const unsigned b2 = __ballot_sync(0xFFFFFFFFu, eopen);
            const unsigned b3 = __ballot_sync(0xFFFFFFFFu, fopen);
            if (lane < 4) {
                const unsigned v = lane == 0 ? b0 : lane == 1 ? b1 : lane == 2 ? b2 : b3;
                dirs[((long long)i * nch + c) * 4 + lane] = v;
            }
            if (i == la && valid && j == lb) final_h = H;
            __syncwarp();
        }
    }
    final_h = __reduce_max_sync(0xFFFFFFFFu, final_h);
    __syncwarp();
    // walk back (lane 0)
    int nr = 0;
    bool ok = final_h == r.score1;
    if (lane == 0 && ok) {
        int i = la, j = lb, state = 0, cur = -1, len = 0, guard = 2 * (la + lb) + 4;
        while ((i > 0 || j > 0) && guard-- > 0) {
            const int off = j - i - dlo;
            if (i < 0 || j < 0 || off < 0 || off >= nch * 32) { ok = false; break; }
            const long long base = ((long long)i * nch + (off >> 5)) * 4;
            const int l = off & 31;
            const int src = ((dirs[base] >> l) & 1) | (((dirs[base + 1] >> l) & 1) << 1);
            const int eo = (dirs[base + 2] >> l) & 1, fo = (dirs[base + 3] >> l) & 1;
            int op;
            if (state == 0) {
                if (src == 0) {
                    op = GSW_CIGAR_M;
                    i--;
                    j--;
                } else {
                    state = src;
                    continue;
                }
            } else if (state == 1) {
                op = GSW_CIGAR_D;
                state = eo ? 0 : 1;
                j--;
            } else {
                op = GSW_CIGAR_I;
                state = fo ? 0 : 2;
                i--;
            }
            if (op == cur) {
                len++;
            } else {
                if (len) ops[nr++] = ((uint32_t)len << 4) | (uint32_t)cur;
                cur = op;
                len = 1;
            }
        }
        if (i != 0 || j != 0) ok = false;
        if (len) ops[nr++] = ((uint32_t)len << 4) | (uint32_t)cur;
    }
    ok = __shfl_sync(0xFFFFFFFFu, (int)ok, 0);
    nr = __shfl_sync(0xFFFFFFFFu, nr, 0);
    gsw_result *rp = b.res + p;
    if (!ok) {
        if (lane == 0) rp->flags |= kResInternal;
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
        }
        return;
    }
    __syncwarp();
    for (int t = lane; t < nr; t += 32) b.cigar[off + t] = ops[nr - 1 - t];
    if (lane == 0) {
        rp->cigar_len = nr;
        rp->cigar_off = (int64_t)off;
        rp->flags &= ~kResPendingTrace;
    }
}

// Persistent: warps take pairs from a counter.  Pairs whose needs fit the
// shared-memory area run there; the others use the warp's global scratch.
__global__ void __launch_bounds__(kTBlock) k_traceback(BatchView b, Scoring sc, TraceScratch ts, TraceCfg cfg) {
    extern __shared__ __align__(16) uint32_t tsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (kTBlock / 32) + warp;
    const int per_warp = cfg.smem_dir_words + cfg.smem_op_words + 2 * 32 * cfg.smem_state_chunks;
    uint32_t *sdir = tsm + (size_t)warp * per_warp;
    uint32_t *sops = sdir + cfg.smem_dir_words;
    int *sst = reinterpret_cast<int *>(sops + cfg.smem_op_words);
    uint32_t *gdir = ts.dirs + (size_t)gwarp * ts.dir_words;
    uint32_t *gops = ts.ops + (size_t)gwarp * ts.op_words;  // ops, then the chunk state
    // the planned list (sorted by cost, descending) is dealt round-robin
    const int first = ts.var_start[5], last = ts.var_start[6];
    const int nwarps = gridDim.x * (kTBlock / 32);
    for (int idx = first + gwarp; idx < last; idx += nwarps) {
        const int p = ts.order[idx];
        const gsw_result r = b.res[p];
        if (!wants_trace(r)) continue;
        Need nd = pair_need(r, sc);
        nd.nch = nd.nch < 0 ? -nd.nch : (dhi_width_chunks(nd));
        const bool small = nd.dir <= cfg.smem_dir_words && nd.ops <= cfg.smem_op_words &&
                           nd.nch <= cfg.smem_state_chunks;
        if (small) {
            trace_pair(b, sc, p, r, nd, sdir, sops, sst, sst + 32 * nd.nch, lane);
        } else if (nd.dir <= ts.dir_words && nd.ops + 2LL * 32 * nd.nch <= ts.op_words) {
            int *st = reinterpret_cast<int *>(gops + nd.ops);
            trace_pair(b, sc, p, r, nd, gdir, gops, st, st + 32 * nd.nch, lane);
        } else {
            if (lane == 0) b.res[p].flags |= kResInternal;  // scratch sized too small: host bug
        }
        __syncwarp();
    }
}


// ---------------------------------------------------------------------------
// Anti-diagonal warp traceback for bands of up to 64*NCH diagonals.
//
// Lane l of chunk c owns diagonals d0 = dlo + 64c + 2l and d0 + 1.  On
// anti-diagonal a = i + j exactly one of them holds a cell, and which one
// ((a - dlo) even: d0) is the same for every lane, so all 32 lanes work every
// step.  The left neighbour (i, j-1) and the upper one (i-1, j) lie on the
// previous anti-diagonal, one diagonal away: either the lane's own other
// diagonal or a neighbour lane's (one shuffle), and the diagonal neighbour is
// the lane's own value from two steps back.  Decision bits: 4 ballots per
// chunk and step.
template <int NCH>
__device__ void trace_ad_pair(const BatchView &b, const Scoring &sc, const int8_t *sW, int p, const gsw_result &r,
                              int dlo, int dhi, uint32_t *dirs, uint32_t *ops, uint4 *stage, int lane) {
    const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
    const uint8_t *qs = b.q + b.q_off[p] + r.read_begin1;
    const uint8_t *ts = b.t + b.t_off[p] + r.ref_begin1;
    const int O = sc.O, X = sc.X, A = sc.A;
    int H1[NCH], E1[NCH], F1[NCH], H2[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) { H1[c] = kNegT; E1[c] = kNegT; F1[c] = kNegT; H2[c] = kNegT; }
    int final_h = kNegT;
    const int steps = la + lb;
    for (int a = 0; a <= steps; a++) {
        const int par = (a - dlo) & 1;
        // neighbour values from the previous anti-diagonal (before any update)
        int nh[NCH], nx[NCH];  // par 0: left (H, E); par 1: up (H, F)
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            if (par == 0) {
                int h = __shfl_up_sync(0xFFFFFFFFu, H1[c], 1), e = __shfl_up_sync(0xFFFFFFFFu, E1[c], 1);
                const int ph = c > 0 ? __shfl_sync(0xFFFFFFFFu, H1[c > 0 ? c - 1 : 0], 31) : kNegT;
                const int pe = c > 0 ? __shfl_sync(0xFFFFFFFFu, E1[c > 0 ? c - 1 : 0], 31) : kNegT;
                nh[c] = lane == 0 ? ph : h;
                nx[c] = lane == 0 ? pe : e;
            } else {
                int h = __shfl_down_sync(0xFFFFFFFFu, H1[c], 1), f = __shfl_down_sync(0xFFFFFFFFu, F1[c], 1);
                const int uh = c + 1 < NCH ? __shfl_sync(0xFFFFFFFFu, H1[c + 1 < NCH ? c + 1 : c], 0) : kNegT;
                const int uf = c + 1 < NCH ? __shfl_sync(0xFFFFFFFFu, F1[c + 1 < NCH ? c + 1 : c], 0) : kNegT;
                nh[c] = lane == 31 ? uh : h;
                nx[c] = lane == 31 ? uf : f;
            }
        }
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            const int d = dlo + 64 * c + 2 * lane + par;
            const int i = (a - d) >> 1, j = (a + d) >> 1;
            const bool valid = d <= dhi && i >= 0 && i <= la && j >= 0 && j <= lb;
            int hl, el, hu, fu;
            if (par == 0) { hl = nh[c]; el = nx[c]; hu = H1[c]; fu = F1[c]; }
            else { hl = H1[c]; el = E1[c]; hu = nh[c]; fu = nx[c]; }
            int E = kNegT, F = kNegT, hdg = kNegT, H;
            bool eopen = false, fopen = false;
            if (j >= 1) {
                const int eo = hl - O;
                E = max(eo, el - X);
                eopen = E == eo;
            }
            if (i >= 1) {
                const int fo = hu - O;
                F = max(fo, fu - X);
                fopen = F == fo;
            }
            if (valid && i >= 1 && j >= 1) {
                const int qa = min((int)qs[i - 1], A - 1), tb = min((int)ts[j - 1], A - 1);
                hdg = H2[c] + sW[qa * A + tb];
            }
            H = max(hdg, max(E, F));
            if (i == 0 && j == 0) H = 0;
            if (!valid || H < kNegHalf) { H = kNegT; E = kNegT; F = kNegT; }
            const int src = (valid && i >= 1 && j >= 1 && hdg > kNegHalf && H == hdg) ? 0 : (H == E ? 1 : 2);
            const unsigned b0 = __ballot_sync(0xFFFFFFFFu, src & 1);
            const unsigned b1 = __ballot_sync(0xFFFFFFFFu, src & 2);
            const unsigned b2 = __ballot_sync(0xFFFFFFFFu, eopen);
            const unsigned b3 = __ballot_sync(0xFFFFFFFFu, fopen);
            if (lane < 4) dirs[((long long)a * NCH + c) * 4 + lane] = lane == 0 ? b0 : lane == 1 ? b1 : lane == 2 ? b2 : b3;
            if (valid && i == la && j == lb) final_h = H;
            H2[c] = H1[c];
            H1[c] = H;
            E1[c] = E;
            F1[c] = F;
        }
    }
    final_h = __reduce_max_sync(0xFFFFFFFFu, final_h);
    __syncwarp();
    gsw_result *rp = b.res + p;
    // Walk back from (la, lb).  The anti-diagonal index i + j never increases
    // along the walk, so the warp stages the decision planes into shared
    // memory 32 anti-diagonals at a time (coalesced) and lane 0 walks inside
    // the staged block; the runs go to `ops` in reverse order.
    constexpr int KB = 32;
    const uint4 *dirs4 = reinterpret_cast<const uint4 *>(dirs);
    int i = la, j = lb, state = 0, cur = -1, len = 0, runs = 0;
    bool ok = final_h == r.score1;
    int a_hi = la + lb;
    while (ok && (i > 0 || j > 0) && a_hi >= 0) {
        const int a_lo = max(0, a_hi - KB + 1);
        const int nwords = (a_hi - a_lo + 1) * NCH;
        for (int w = lane; w < nwords; w += 32) stage[w] = dirs4[(long long)a_lo * NCH + w];
        __syncwarp();
        if (lane == 0) {
            while ((i > 0 || j > 0) && i + j >= a_lo) {
                const int off2 = j - i - dlo;
                if (i < 0 || j < 0 || off2 < 0 || off2 >= 64 * NCH) { ok = false; break; }
                const uint4 pl = stage[(i + j - a_lo) * NCH + (off2 >> 6)];
                const int l = (off2 & 63) >> 1;
                const int src = ((pl.x >> l) & 1) | (((pl.y >> l) & 1) << 1);
                const int eo = (pl.z >> l) & 1, fo = (pl.w >> l) & 1;
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
        a_hi = a_lo - 1;
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
    __shared__ uint4 stage_all[kTBlock / 32][32 * NCH];
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
        if ((long long)(la + lb + 1) * NCH * 4 > ts.dir_words || dhi - dlo + 1 > 64 * NCH ||
            (long long)(la + lb + 2) > ts.op_words) {
            if (lane == 0) b.res[p].flags |= kResInternal;
            continue;
        }
        trace_ad_pair<NCH>(b, sc, sW, p, r, dlo, dhi, dirs, ops, stage_all[warp], lane);
    }
}

}  // namespace

// classes of the warp traceback: 0..3 = anti-diagonal kernel with 1/2/4/8
// chunks of 64 diagonals, 4 = the row kernel (wider bands)
int trace_class(int width) {
    return width <= 64 ? 0 : width <= 128 ? 1 : width <= 256 ? 2 : width <= 512 ? 3 : 4;
}

cudaError_t launch_trace_ad(const BatchView &b, const Scoring &sc, const TraceScratch &ts, int grid,
                            cudaStream_t st) {
    k_trace_ad<1><<<grid, kTBlock, 0, st>>>(b, sc, ts, 0);
    k_trace_ad<2><<<grid, kTBlock, 0, st>>>(b, sc, ts, 1);
    k_trace_ad<4><<<grid, kTBlock, 0, st>>>(b, sc, ts, 2);
    k_trace_ad<8><<<grid, kTBlock, 0, st>>>(b, sc, ts, 3);
    return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------------------
// Wide anti-diagonal traceback (bands of 513 .. 64*kAdwMaxChunks diagonals,
// long reads): the same wavefront as k_trace_ad, with each chunk's state
// (H, E, F of the previous anti-diagonal, H of the one before) in shared
// memory.  Chunks are visited in descending order on even steps (each needs
// its left neighbour chunk's old value) and ascending order on odd steps (its
// right neighbour's), so no chunk is read after it was updated in the same
// step.  One warp per block; the walk stages 16 anti-diagonals at a time.
constexpr int kAdwStage = 16;

__device__ void trace_adw_pair(const BatchView &b, const Scoring &sc, const int8_t *sW, int p, const gsw_result &r,
                               int dlo, int dhi, int nch, uint32_t *dirs, uint32_t *ops, int4 *state, uint4 *stage,
                               int lane) {
    const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
    const uint8_t *qs = b.q + b.q_off[p] + r.read_begin1;
    const uint8_t *ts = b.t + b.t_off[p] + r.ref_begin1;
    const int O = sc.O, X = sc.X, A = sc.A;
    for (int c = 0; c < nch; c++) state[c * 32 + lane] = make_int4(kNegT, kNegT, kNegT, kNegT);
    __syncwarp();
    int final_h = kNegT;
    const int steps = la + lb;
    for (int a = 0; a <= steps; a++) {
        const int par = (a - dlo) & 1;
        for (int t = 0; t < nch; t++) {
            const int c = par == 0 ? nch - 1 - t : t;
            const int4 stv = state[c * 32 + lane];  // x: H1, y: E1, z: F1, w: H2
            int hl, el, hu, fu;
            if (par == 0) {
                int h = __shfl_up_sync(0xFFFFFFFFu, stv.x, 1), e = __shfl_up_sync(0xFFFFFFFFu, stv.y, 1);
                if (lane == 0) {
                    if (c > 0) {
                        const int4 nb = state[(c - 1) * 32 + 31];
                        h = nb.x;
                        e = nb.y;
                    } else {
                        h = kNegT;
                        e = kNegT;
                    }
                }
                hl = h; el = e; hu = stv.x; fu = stv.z;
            } else {
                int h = __shfl_down_sync(0xFFFFFFFFu, stv.x, 1), f = __shfl_down_sync(0xFFFFFFFFu, stv.z, 1);
                if (lane == 31) {
                    if (c + 1 < nch) {
                        const int4 nb = state[(c + 1) * 32];
                        h = nb.x;
                        f = nb.z;
                    } else {
                        h = kNegT;
                        f = kNegT;
                    }
                }
                hl = stv.x; el = stv.y; hu = h; fu = f;
            }
            __syncwarp();
            const int d = dlo + 64 * c + 2 * lane + par;
            const int i = (a - d) >> 1, j = (a + d) >> 1;
            const bool valid = d <= dhi && i >= 0 && i <= la && j >= 0 && j <= lb;
            int E = kNegT, F = kNegT, hdg = kNegT, H;
            bool eopen = false, fopen = false;
            if (j >= 1) {
                const int eo = hl - O;
                E = max(eo, el - X);
                eopen = E == eo;
            }
            if (i >= 1) {
                const int fo = hu - O;
                F = max(fo, fu - X);
                fopen = F == fo;
            }
            if (valid && i >= 1 && j >= 1) {
                const int qa = min((int)qs[i - 1], A - 1), tb = min((int)ts[j - 1], A - 1);
                hdg = stv.w + sW[qa * A + tb];
            }
            H = max(hdg, max(E, F));
            if (i == 0 && j == 0) H = 0;
            if (!valid || H < kNegHalf) { H = kNegT; E = kNegT; F = kNegT; }
            const int src = (valid && i >= 1 && j >= 1 && hdg > kNegHalf && H == hdg) ? 0 : (H == E ? 1 : 2);
            const unsigned b0 = __ballot_sync(0xFFFFFFFFu, src & 1);
            const unsigned b1 = __ballot_sync(0xFFFFFFFFu, src & 2);
            const unsigned b2 = __ballot_sync(0xFFFFFFFFu, eopen);
            const unsigned b3 = __ballot_sync(0xFFFFFFFFu, fopen);
            if (lane < 4) dirs[((long long)a * nch + c) * 4 + lane] = lane == 0 ? b0 : lane == 1 ? b1 : lane == 2 ? b2 : b3;
            if (valid && i == la && j == lb) final_h = H;
            state[c * 32 + lane] = make_int4(H, E, F, stv.x);
            __syncwarp();
        }
    }
    final_h = __reduce_max_sync(0xFFFFFFFFu, final_h);
    __syncwarp();
    gsw_result *rp = b.res + p;
    const uint4 *dirs4 = reinterpret_cast<const uint4 *>(dirs);
    int i = la, j = lb, state_w = 0, cur = -1, len = 0, runs = 0;
    bool ok = final_h == r.score1;
    int a_hi = la + lb;
    while (ok && (i > 0 || j > 0) && a_hi >= 0) {
        const int a_lo = max(0, a_hi - kAdwStage + 1);
        const int nwords = (a_hi - a_lo + 1) * nch;
        for (int w = lane; w < nwords; w += 32) stage[w] = dirs4[(long long)a_lo * nch + w];
        __syncwarp();
        if (lane == 0) {
            while ((i > 0 || j > 0) && i + j >= a_lo) {
                const int off2 = j - i - dlo;
                if (i < 0 || j < 0 || off2 < 0 || off2 >= 64 * nch) { ok = false; break; }
                const uint4 pl = stage[(i + j - a_lo) * nch + (off2 >> 6)];
                const int l = (off2 & 63) >> 1;
                const int src = ((pl.x >> l) & 1) | (((pl.y >> l) & 1) << 1);
                const int eo = (pl.z >> l) & 1, fo = (pl.w >> l) & 1;
                int op;
                if (state_w == 0) {
                    if (src == 0) { op = GSW_CIGAR_M; i--; j--; }
                    else { state_w = src; continue; }
                } else if (state_w == 1) {
                    op = GSW_CIGAR_D; state_w = eo ? 0 : 1; j--;
                } else {
                    op = GSW_CIGAR_I; state_w = fo ? 0 : 2; i--;
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
        a_hi = a_lo - 1;
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

__global__ void __launch_bounds__(32) k_trace_adw(BatchView b, Scoring sc, TraceScratch ts, int cls, int nch_max) {
    extern __shared__ __align__(16) uint8_t adw_smem[];
    __shared__ int8_t sW[kMaxAlpha * kMaxAlpha];
    for (int i = threadIdx.x; i < sc.A * sc.A; i += blockDim.x) sW[i] = sc.W[i];
    __syncwarp();
    int4 *state = reinterpret_cast<int4 *>(adw_smem);
    uint4 *stage = reinterpret_cast<uint4 *>(adw_smem + (size_t)nch_max * 32 * sizeof(int4));
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x;
    const int nwarps = gridDim.x;
    uint32_t *dirs = ts.dirs + (size_t)gwarp * ts.dir_words;
    uint32_t *ops = ts.ops + (size_t)gwarp * ts.op_words;
    const int first = ts.var_start[cls], last = ts.var_start[cls + 1];
    for (int idx = first + gwarp; idx < last; idx += nwarps) {
        const int p = ts.order[idx];
        const gsw_result r = b.res[p];
        if (!wants_trace(r)) continue;
        const int la = r.read_end1 - r.read_begin1 + 1, lb = r.ref_end1 - r.ref_begin1 + 1;
        int dlo, dhi;
        const int width = band_range(la, lb, r.score1, sc, &dlo, &dhi);
        const int nch = (width + 63) / 64;
        if (nch > nch_max || (long long)(la + lb + 1) * nch * 4 > ts.dir_words || (long long)(la + lb + 2) > ts.op_words) {
            if (lane == 0) b.res[p].flags |= kResInternal;
            continue;
        }
        trace_adw_pair(b, sc, sW, p, r, dlo, dhi, nch, dirs, ops, state, stage, lane);
    }
}

}  // namespace

size_t trace_adw_smem(int nch_max) { return (size_t)nch_max * 32 * sizeof(int4) + (size_t)kAdwStage * nch_max * sizeof(uint4); }
int trace_adw_max_chunks() { return kAdwMaxChunks; }

cudaError_t launch_trace_adw(const BatchView &b, const Scoring &sc, const TraceScratch &ts, int grid, int nch_max,
                             cudaStream_t st) {
    const size_t smem = trace_adw_smem(nch_max);
    cudaFuncSetAttribute(k_trace_adw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_trace_adw<<<grid, 32, smem, st>>>(b, sc, ts, 4, nch_max);
    return cudaGetLastError();
}

namespace {
}  // namespace

int trace_block_threads() { return kTBlock; }

// Maximum needs over the batch: [0] direction words, [1] op words, [2] chunks.
cudaError_t launch_trace_need(const BatchView &b, const Scoring &sc, unsigned long long *max_need,
                              cudaStream_t st) {
    cudaMemsetAsync(max_need, 0, 9 * sizeof(unsigned long long), st);
    const int nb = (b.npairs + 255) / 256;
    if (nb > 0) k_trace_need<<<nb, 256, 0, st>>>(b, sc, max_need);
    return cudaGetLastError();
}

static TraceCfg trace_cfg() { return TraceCfg{4096, 1024, 4}; }

size_t trace_smem_bytes() {
    const TraceCfg c = trace_cfg();
    return (size_t)(c.smem_dir_words + c.smem_op_words + 2 * 32 * c.smem_state_chunks) * 4 * (kTBlock / 32);
}

cudaError_t launch_traceback(const BatchView &b, const Scoring &sc, const TraceScratch &ts, int grid,
                             cudaStream_t st) {
    const size_t smem = trace_smem_bytes();
    cudaFuncSetAttribute(k_traceback, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_traceback<<<grid, kTBlock, smem, st>>>(b, sc, ts, trace_cfg());
    return cudaGetLastError();
}

}  // namespace gsw
