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
    const int w = band_halfwidth(la, lb, r.score1, sc);
    const int delta = lb - la;
    int dlo = min(0, delta) - w, dhi = max(0, delta) + w;
    dlo = max(dlo, -la);
    dhi = min(dhi, lb);
    nd.dlo = dlo;
    nd.dhi = dhi;
    nd.nch = (dhi - dlo + 32) / 32;
    nd.dir = (long long)(la + 1) * nd.nch * 4;
    nd.ops = (long long)la + lb + 2;
    return nd;
}

// pairs the thread-per-pair band kernel left to this kernel (band too wide)
__device__ __forceinline__ bool wants_trace(const gsw_result &r) {
    return r.score1 > 0 && (r.flags & kResPendingTrace) && !(r.flags & kResInternal) && r.read_begin1 >= 0 &&
           r.ref_begin1 >= 0;
}

__global__ void k_trace_need(BatchView b, Scoring sc, unsigned long long *max_need) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned d = 0, o = 0, c = 0;
    if (p < b.npairs) {
        const gsw_result r = b.res[p];
        if (wants_trace(r)) {
            const Need nd = pair_need(r, sc);
            d = (unsigned)min(nd.dir, (long long)UINT_MAX);
            o = (unsigned)min(nd.ops, (long long)UINT_MAX);
            c = (unsigned)nd.nch;
        }
    }
    d = __reduce_max_sync(0xFFFFFFFFu, d);
    o = __reduce_max_sync(0xFFFFFFFFu, o);
    c = __reduce_max_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0 && c > 0) {
        atomicMax(&max_need[0], (unsigned long long)d);
        atomicMax(&max_need[1], (unsigned long long)o);
        atomicMax(&max_need[2], (unsigned long long)c);
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
    const int first = ts.var_start[0], last = ts.var_start[1];
    const int nwarps = gridDim.x * (kTBlock / 32);
    for (int idx = first + gwarp; idx < last; idx += nwarps) {
        const int p = ts.order[idx];
        const gsw_result r = b.res[p];
        if (!wants_trace(r)) continue;
        const Need nd = pair_need(r, sc);
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

}  // namespace

int trace_block_threads() { return kTBlock; }

// Maximum needs over the batch: [0] direction words, [1] op words, [2] chunks.
cudaError_t launch_trace_need(const BatchView &b, const Scoring &sc, unsigned long long *max_need,
                              cudaStream_t st) {
    cudaMemsetAsync(max_need, 0, 3 * sizeof(unsigned long long), st);
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
