// Local Smith-Waterman-Gotoh fill on sm_103a: the hot loop of the method
// ("Algorithm and implementation", item (1): fill the score matrix while
// keeping the per-column "max" array and the column holding the matrix
// maximum; item (2): the suboptimal score from the masked max array).
//
// Layout ("folded ring").  One pair is handled by a group of P consecutive
// lanes of a warp.  A strip of 2*P*R query rows is split into a low half
// (rows [0, S)) and a high half (rows [S, 2S)), S = P*R.  Lane k owns R
// 32-bit words; word r packs low-half row k*R + r in bits 0-15 and high-half
// row S + k*R + r in bits 16-31, each as (value + 0x8000).  Per step, lane k
// computes its R words for target column j = step - k in the low half and
// column j - P in the high half, then passes its bottom row (H, F) and the
// running column maximum to lane k+1 by a shuffle; lane P-1 passes its low
// half to lane 0, whose high half continues that column P steps later.  So
// every cell update is one lane of a 16x2 word, and the recurrences run on
// full-rate instructions only:
//     H  = max(H(i-1,j-1) + W, E, 0, F)      (IADD, 3x VIMNMX.U16x2)
//     m  = max(m, H)                          (column max, VIMNMX)
//     E' = max(E - X, H - O),  F' = max(F - X, H - O)   (2 IADD + 2 VIMNMX + IADD)
// Adds are exact per lane because every lane value stays in [0, 0xFFFF] as
// long as no score exceeds 32767 - max W; a pair whose maximum does is
// flagged and re-filled in 32-bit lanes (same ring, one row per word).
//
// The score lookup W(q_i, t_j) comes from a shared-memory profile: for DNA (4
// letters) one word per (row pair, low letter, high letter), i.e. 16 x R words
// per lane; for other alphabets one low table and one high table.  The words
// of the 32 lanes of a warp are interleaved (lane-minor, 16-byte vectors), so
// the vector loads of a warp never collide in a bank although every lane reads
// a different letter pair.
//
// Critical path.  With O >= X, max(F - X, H - O) = max(F - X, T - O) where
// T = max(H(i-1,j-1) + W, E, 0) does not depend on F, so the F chain down a
// lane's rows is one add and one max per row.
//
// End position (the paper's "recorded column"): every lane tracks, per half,
// the first column where its running column maximum (the maximum over rows 0
// .. its last row) strictly improved, and keeps a copy of its own rows of that
// column.  The lane-(P-1) high-half tracker gives score1 and the end column;
// the first lane/half whose tracker holds (score1, end column) holds the end
// row in its saved copy.
#include "gsw_impl.cuh"

#include <climits>

#include <type_traits>
#include <cstring>
#include <mutex>

namespace gsw {
namespace {

constexpr int kBlock = 128;
constexpr int kUnrollFast = 4;  // steady loop of one-strip forward fills
// The steady forward steps (FAST, FwdFirst, FwdLater) of 16-bit lanes keep
// the tracker's two columns as the signed 16-bit halves of one word: targets
// up to this many columns take them
constexpr int kFastMaxCols = 32768;
constexpr int kUnrollGen = 4;   // other steady loops
// forms of the strip step (StripRunner::step)
constexpr int kModeGen = 0, kModeFast = 1, kModeFwdFirst = 2, kModeFwdLater = 3, kModeRev = 4;

// ---------------------------------------------------------------- lanes
struct L16 {
    static constexpr bool FOLD = true;
    using cm_t = uint16_t;
    using bnd_t = uint32_t;
    // lane values are biased by 0x8000 in unsigned 16-bit halves (measured
    // against signed halves with the zero clamp folded into a DPX add-max:
    // one instruction fewer per word but one DPX more, slower)
    static constexpr uint32_t Z = 0x8000u;    // bias of one lane
    static constexpr uint32_t Z2 = 0x80008000u;
    static __device__ __forceinline__ uint32_t vmax(uint32_t a, uint32_t b) { return __vmaxu2(a, b); }
    static __device__ __forceinline__ uint32_t lane1(int v) { return (uint32_t)(v + 0x8000) & 0xFFFFu; }
    static __device__ __forceinline__ uint32_t cm16(uint32_t x) { return x; }
    static __device__ __forceinline__ int value(uint32_t x16) { return (int)x16 - 0x8000; }
    static __device__ __forceinline__ uint32_t tt_relu(uint32_t d, uint32_t w, uint32_t e) {
        return vmax(addmax(d, w, e), Z2);
    }
    // H - O per lane: a plain add (every biased lane value is >= O)
    static __device__ __forceinline__ uint32_t ok(int O) { return addk(-O); }
    static __device__ __forceinline__ uint32_t sub_o(uint32_t h, uint32_t kO) { return h + kO; }
    static __device__ __forceinline__ uint32_t both(int v) { return lane1(v) | (lane1(v) << 16); }
    // integer that adds c to both lanes of a word
    static __device__ __forceinline__ uint32_t addk(int c) { return (uint32_t)(c * 65537); }
    // per-lane max(a + b, c) in one DPX instruction; b holds two 16-bit
    // two's-complement halves (no borrow between them)
    static __device__ __forceinline__ uint32_t addmax(uint32_t a, uint32_t b, uint32_t c) {
        return __viaddmax_u16x2(a, b, c);
    }
    static __device__ __forceinline__ uint32_t halves(int lo, int hi) {
        return ((uint32_t)lo & 0xFFFFu) | (((uint32_t)hi & 0xFFFFu) << 16);
    }
    // low half of a, high half of b (words made by halves)
    static __device__ __forceinline__ uint32_t merge(uint32_t a, uint32_t b) {
        return (a & 0x0000FFFFu) | (b & 0xFFFF0000u);
    }
};

struct L32 {
    static constexpr bool FOLD = false;
    using cm_t = int32_t;
    using bnd_t = int2;
    static constexpr uint32_t Z = 0u;
    static constexpr uint32_t Z2 = 0u;
    static __device__ __forceinline__ uint32_t vmax(uint32_t a, uint32_t b) {
        return (uint32_t)max((int)a, (int)b);
    }
    static __device__ __forceinline__ uint32_t lane1(int v) { return (uint32_t)v; }
    static __device__ __forceinline__ uint32_t both(int v) { return (uint32_t)v; }
    static __device__ __forceinline__ uint32_t addk(int c) { return (uint32_t)c; }
    static __device__ __forceinline__ uint32_t addmax(uint32_t a, uint32_t b, uint32_t c) { return vmax(a + b, c); }
    static __device__ __forceinline__ uint32_t halves(int lo, int hi) { return (uint32_t)lo; }
    static __device__ __forceinline__ uint32_t merge(uint32_t a, uint32_t b) { return a; }
    static __device__ __forceinline__ uint32_t cm16(uint32_t x) { return x; }
    static __device__ __forceinline__ uint32_t tt_relu(uint32_t d, uint32_t w, uint32_t e) {
        return vmax(addmax(d, w, e), Z2);
    }
    static __device__ __forceinline__ uint32_t ok(int O) { return addk(-O); }
    static __device__ __forceinline__ uint32_t sub_o(uint32_t h, uint32_t kO) { return h + kO; }
};

// Words of one lane's profile (the warp region holds 32 lanes' worth).  DNA
// in 16-bit lanes: a low-letter table and a high-letter table (8 R words),
// added per step (measured against one word per letter pair, 16 R words,
// whose larger profile costs occupancy, and one table holding both halves,
// 4 R words, merged by a logic op that issues at a lower rate than the add:
// both slower); other alphabets: one table with both halves per letter.
__host__ __device__ constexpr int prof_words(int R, bool fold, bool dna, int A) {
    return dna ? (fold ? 8 * R : 4 * R) : A * R;
}

// Index of profile word (table c, row r) of lane l inside the warp region:
// lane-minor groups of 4, 2 or 1 consecutive rows (the vector width).
template <int R>
__device__ __forceinline__ int pidx(int c, int r, int l) {
    if constexpr (R % 4 == 0) return ((c * (R / 4) + r / 4) * 32 + l) * 4 + (r & 3);
    else if constexpr (R % 2 == 0) return ((c * (R / 2) + r / 2) * 32 + l) * 2 + (r & 1);
    else return (c * R + r) * 32 + l;
}

// One fill job for a group (one pair).
struct Job {
    const uint8_t *q;  // query row i at q[i * qs]
    int qs;
    int mrows;
    const uint8_t *t;  // target column j at t[j * ts]
    int ts;
    int ncols;
    uint32_t stop_u;   // reverse mode: stop at the first full column whose max equals this (biased); 0 = never
    void *cms;         // column-max scratch (ncols entries)
    void *bnd;         // strip boundary scratch (2 x ncols entries, ping-pong)
};

struct RingResult {
    int score;  // max over the matrix (>= 0)
    int col;    // first column reaching it (-1 if score == 0)
    int row;    // first row of that column holding it, in padded row space
    int pad_top;
};

// Loads the R words of table c for lane l.
template <int R>
__device__ __forceinline__ void load_words(const uint32_t *base, int c, int l, uint32_t (&w)[R]) {
    if constexpr (R % 4 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(base + pidx<R>(c, r, l));
            w[r] = v.x; w[r + 1] = v.y; w[r + 2] = v.z; w[r + 3] = v.w;
        }
    } else if constexpr (R % 2 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            const uint2 v = *reinterpret_cast<const uint2 *>(base + pidx<R>(c, r, l));
            w[r] = v.x; w[r + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; r++) w[r] = base[pidx<R>(c, r, l)];
    }
}

__device__ __forceinline__ int sc_w(const Scoring &sc, int a, int b) { return sc.W[a * sc.A + b]; }

// Builds this lane's profile for strip `st` (padded rows of the strip:
// [st*SP, st*SP + SP); padded row rho holds query row rho - pad_top).
template <int P, int R, class L, bool DNA>
__device__ __forceinline__ void build_profile(uint32_t *psm, const Job &job, const Scoring &sc, int k, int lane,
                                              int st, int pad_top) {
    constexpr int S = P * R;
    constexpr int SP = L::FOLD ? 2 * S : S;
    const int A = sc.A;
#pragma unroll 1
    for (int r = 0; r < R; r++) {
        int rho_lo = st * SP + k * R + r - pad_top;
        int qlo = rho_lo >= 0 ? min((int)job.q[(long long)rho_lo * job.qs], A - 1) : -1;
        int qhi = -1;
        if constexpr (L::FOLD) {
            int rho_hi = st * SP + S + k * R + r - pad_top;
            qhi = rho_hi >= 0 ? min((int)job.q[(long long)rho_hi * job.qs], A - 1) : -1;
        }
        if constexpr (DNA) {
            for (int a = 0; a < A; a++) {
                psm[pidx<R>(a, r, lane)] = L::halves(qlo >= 0 ? sc_w(sc, qlo, a) : 0, 0);
                if constexpr (L::FOLD)
                    psm[pidx<R>(A + a, r, lane)] = L::halves(0, qhi >= 0 ? sc_w(sc, qhi, a) : 0);
            }
        } else {
            // general alphabets: one table, both halves' scores in one word
            // (the step takes the low half from the low letter's word and the
            // high half from the high letter's), half the shared memory of
            // two tables
            for (int a = 0; a < A; a++)
                psm[pidx<R>(a, r, lane)] =
                    L::halves(qlo >= 0 ? sc_w(sc, qlo, a) : 0, L::FOLD && qhi >= 0 ? sc_w(sc, qhi, a) : 0);
        }
    }
}

template <class L>
__device__ __forceinline__ int lane_lo(uint32_t w) {
    if constexpr (L::FOLD) return L::value(w & 0xFFFFu);
    else return (int)w;
}
template <class L>
__device__ __forceinline__ int lane_hi(uint32_t w) {
    if constexpr (L::FOLD) return L::value(w >> 16);
    else return (int)w;
}

// One strip of the ring fill for the P lanes of a group: the per-strip state
// (H, E, the saved column, the trackers, the values received from the lane
// above) and the step.  ring_fill runs the strips of a pair one after the
// other; k_fill_long runs them on several warps of a CTA at once.
template <int P, int R, class L, bool DNA>
struct StripRunner {
    static constexpr int S = P * R;
    static constexpr int SP = L::FOLD ? 2 * S : S;
    static constexpr uint32_t Z2 = L::Z2;
    using bnd_t = typename L::bnd_t;
    using cm_t = typename L::cm_t;
    static constexpr int CM_OFF = L::FOLD ? -(2 * P - 1) : -(P - 1);

    Job job;
    uint32_t *psm;
    int k, gbase, lane, src, n, A, nsteps, pad_top;
    unsigned gmask;
    uint32_t kO, kXm, NEGE;
    uint32_t bzh, bzf, bzc;
    uint32_t mulh;  // received word -> this lane's input: lane 0 shifts it to the high half (x 65536)
    cm_t *cms;
    bool has_cms;

    // Binds the runner to a pair (job) and to lane k of the group at gbase.
    __device__ __forceinline__ void init(const Job &job_, const Scoring &sc, uint32_t *psm_, int k_, unsigned gmask_,
                                         int gbase_, int lane_, int pad_top_) {
        job = job_;
        psm = psm_;
        k = k_;
        gbase = gbase_;
        lane = lane_;
        src = gbase_ + ((k_ + P - 1) & (P - 1));
        n = job_.ncols;
        A = sc.A;
        nsteps = job_.ncols + (L::FOLD ? 2 * P - 1 : P - 1);
        pad_top = pad_top_;
        gmask = gmask_;
        kO = L::ok(sc.O);
        kXm = L::halves(-sc.X, -sc.X);
        NEGE = L::both(-sc.O);
        bzh = k_ == 0 ? L::lane1(0) : 0u;
        bzf = k_ == 0 ? L::lane1(-sc.O) : 0u;
        bzc = k_ == 0 ? (L::FOLD ? L::Z : 0u) : 0u;
        mulh = k_ == 0 ? (L::FOLD ? 65536u : 0u) : 1u;
        cms = reinterpret_cast<cm_t *>(job_.cms);
        has_cms = job_.cms != nullptr;
    }

    int st = 0;
    bool last_strip = false;
    const bnd_t *bin = nullptr;
    bnd_t *bout = nullptr;
    uint32_t H[R], E[R], SV[R];
    uint32_t hdiag, best, xh, xf, xc;
    int c_lo, c_hi, nal, nah;
    uint32_t cpk;  // FAST steps (16-bit lanes): c_lo and c_hi as the halves of one word
    bnd_t b_cur, b_nxt;
    cm_t c_cur, c_nxt;
    uint32_t cmpk, cmw0;  // max-array values of the packed 4-step store


    // Strips after the first read the previous strip's boundary (lane 0,
    // column s) and accumulate the column max (lane P-1, column s-2P+1): the
    // group loads both one block of P columns ahead and the two lanes take
    // their word by shuffle, so no step waits on global memory.
    __device__ __forceinline__ void prefetch(const int s0) {
        const int jb = s0 + k, jc = s0 + CM_OFF + k;
        b_nxt = (jb >= 0 && jb < n) ? bin[jb] : bnd_t{};
        c_nxt = (has_cms && jc >= 0 && jc < n) ? cms[jc] : cm_t{};
    }

    // Starts strip st_ (boundary in from bin_, out to bout_).
    __device__ void begin(const Scoring &sc, int st_, const bnd_t *bin_, bnd_t *bout_, bool last_) {
        st = st_;
        bin = bin_;
        bout = bout_;
        last_strip = last_;
        build_profile<P, R, L, DNA>(psm, job, sc, k, lane, st, pad_top);
        __syncwarp(gmask);
#pragma unroll
        for (int r = 0; r < R; r++) { H[r] = Z2; E[r] = NEGE; SV[r] = Z2; }
        hdiag = Z2;
        best = Z2;
        c_lo = -1;
        c_hi = -1;
        xh = Z2;  // values received from lane k-1
        xf = NEGE;
        xc = Z2;
        nal = (-k >= 0 && -k < n) ? min((int)job.t[0], A - 1) : 0;
        nah = 0;
        b_cur = bnd_t{};
        b_nxt = bnd_t{};
        c_cur = cm_t{};
        c_nxt = cm_t{};
        if (st > 0) prefetch(0);
    }

    // One step of lane k: low half at column s - k, high half P columns
    // behind.  CHECKED steps handle columns outside [0, n) (start-up and
    // drain of the wavefront); steady steps have every column in range.
    // MODE: kModeGen decides everything at run time; the other modes are the
    // steady steps of forward fills with a max array (no reverse stop):
    // kModeFast one strip (no boundary rows), kModeFwdFirst the first of
    // several strips (boundary row out), kModeFwdLater a later strip
    // (boundary row in, the max array merged with the strips above).
    // Returns true when the reverse fill found its target column.
    template <bool CHECKED, int MODE = kModeGen, int PK = -1>
    __device__ __forceinline__ bool step(const int s) {
        constexpr bool FAST = MODE == kModeFast;
        const int jlo = s - k;
        const int jhi = L::FOLD ? jlo - P : jlo;
        uint32_t hin, fin, cmin;
        // lane 0 shifts the received word to its high half (the fold) and
        // puts its boundary in the low half: one multiply-add each, on the
        // FMA pipe that the cell arithmetic leaves mostly idle
        hin = xh * mulh + bzh;
        fin = xf * mulh + bzf;
        cmin = xc * mulh + bzc;
        constexpr bool REV = MODE == kModeRev;
        cm_t cm_prev{};
        if ((MODE == kModeGen || REV) ? st > 0 : MODE == kModeFwdLater) {
            const int bi = s & (P - 1);
            if (bi == 0) {
                b_cur = b_nxt;
                c_cur = c_nxt;
                prefetch(s + P);
            }
            const int srcl = gbase + bi;
            if constexpr (REV) {
                // (no max array)
            } else if constexpr (L::FOLD) {
                cm_prev = (cm_t)__shfl_sync(gmask, (uint32_t)c_cur, srcl);
            } else {
                cm_prev = __shfl_sync(gmask, c_cur, srcl);
            }
            bnd_t w;
            if constexpr (L::FOLD) {
                w = __shfl_sync(gmask, b_cur, srcl);
            } else {
                w.x = __shfl_sync(gmask, b_cur.x, srcl);
                w.y = __shfl_sync(gmask, b_cur.y, srcl);
            }
            if (k == 0 && (!CHECKED || (jlo >= 0 && jlo < n))) {
                if constexpr (L::FOLD) {
                    hin = (hin & 0xFFFF0000u) | (w & 0xFFFFu);
                    fin = (fin & 0xFFFF0000u) | (w >> 16);
                } else {
                    hin = (uint32_t)w.x;
                    fin = (uint32_t)w.y;
                }
            }
        }
        // letters of this lane's columns (loaded one step ahead)
        const int al = nal, ah = nah;
        {
            const int j1 = jlo + 1;
            if constexpr (CHECKED) {
                nal = (j1 >= 0 && j1 < n) ? min((int)job.t[(long long)j1 * job.ts], A - 1) : 0;
                if constexpr (L::FOLD) {
                    const int j2 = j1 - P;
                    nah = (j2 >= 0 && j2 < n) ? min((int)job.t[(long long)j2 * job.ts], A - 1) : 0;
                }
            } else if constexpr (FAST) {
                // letters were checked before the fill (bad_letters, or the
                // static entry's per-pair check): no clamp
                nal = job.t[j1];
                if constexpr (L::FOLD) nah = job.t[j1 - P];
            } else {
                nal = min((int)job.t[(long long)j1 * job.ts], A - 1);
                if constexpr (L::FOLD) nah = min((int)job.t[(long long)(j1 - P) * job.ts], A - 1);
            }
        }
        uint32_t pw[R];
        if constexpr (DNA) {
            load_words<R>(psm, al, lane, pw);
            if constexpr (L::FOLD) {
                uint32_t ph[R];
                load_words<R>(psm, A + ah, lane, ph);
#pragma unroll
                for (int r = 0; r < R; r++) pw[r] += ph[r];
            }
        } else {
            load_words<R>(psm, al, lane, pw);
            if constexpr (L::FOLD) {
                uint32_t ph[R];
                load_words<R>(psm, ah, lane, ph);
#pragma unroll
                for (int r = 0; r < R; r++) pw[r] = L::merge(pw[r], ph[r]);
            }
        }
        uint32_t diag = hdiag;
        hdiag = hin;
        uint32_t f = fin, m = cmin;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const uint32_t tt = L::tt_relu(diag, pw[r], E[r]);
            const uint32_t h = L::vmax(tt, f);
            // one H - O for both gap states; the F chain then runs through
            // h (3 dependent instructions per row), hidden by the other warps
            const uint32_t ho = L::sub_o(h, kO);
            f = L::addmax(f, kXm, ho);
            E[r] = L::addmax(E[r], kXm, ho);
            diag = H[r];
            H[r] = h;
            m = L::vmax(m, h);
        }
        uint32_t cme = m;
        if constexpr (CHECKED) {
            // before a half's first column its state must be the left boundary
            if (jhi < 0) {
                const uint32_t keep = (L::FOLD && jlo >= 0) ? 0x0000FFFFu : 0u;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    H[r] = (H[r] & keep) | (Z2 & ~keep);
                    E[r] = (E[r] & keep) | (NEGE & ~keep);
                }
                hdiag = (hdiag & keep) | (Z2 & ~keep);
            }
            uint32_t vm = 0;
            if (jlo >= 0 && jlo < n) vm |= L::FOLD ? 0x0000FFFFu : 0xFFFFFFFFu;
            if (L::FOLD && jhi >= 0 && jhi < n) vm |= 0xFFFF0000u;
            cme = (m & vm) | (Z2 & ~vm);
        }
        // tracker: first column where the running column max strictly improved
        {
            // branch-free: a mask of the halves that improved selects this
            // column's rows into the saved copy (no branch splits the step,
            // so the steps of the unrolled loop interleave)
            const uint32_t nb = L::vmax(cme, best);
            const uint32_t diff = nb ^ best;
            uint32_t mk;
            if constexpr (L::FOLD) {
                const uint32_t t = __vminu2(diff, 0x00010001u);  // 1 in each half that changed
                mk = t * 0xFFFFu;
                if constexpr (MODE != kModeGen) {
                    // both columns in one word (columns < 2^15 in the
                    // steady forward steps): one multiply-add makes
                    // (jhi, jlo), one logic op takes the halves that improved
                    const uint32_t jpk = (uint32_t)jlo * 0x10001u - ((uint32_t)P << 16);
                    cpk = (jpk & mk) | (cpk & ~mk);
                } else {
                    c_lo = (t & 1u) ? jlo : c_lo;
                    c_hi = (t >> 16) ? jhi : c_hi;
                }
            } else {
                mk = diff ? 0xFFFFFFFFu : 0u;
                c_lo = diff ? jlo : c_lo;
            }
            best = nb;
#pragma unroll
            for (int r = 0; r < R; r++) SV[r] = (H[r] & mk) | (SV[r] & ~mk);
        }

        // the last lane holds complete columns: column max and strip boundary
        bool found = false;
        if (FAST && PK >= 0) {
            // four columns' maxima in one 8-byte store: two 16-bit values per
            // word, packed on the way (jhi of the block's first step is a
            // multiple of 4)
            if constexpr ((PK & 1) == 0) {
                cmpk = m >> 16;
            } else {
                const uint32_t w = cmpk | (m & 0xFFFF0000u);
                if constexpr (PK == 1) cmw0 = w;
                else if (k == P - 1) *reinterpret_cast<uint2 *>(cms + (jhi - 3)) = make_uint2(cmw0, w);
            }
        } else if (FAST && k == P - 1) {
            if constexpr (L::FOLD) cms[jhi] = (uint16_t)L::cm16(m >> 16);
            else cms[jhi] = (int)m;
        } else if ((MODE == kModeFwdFirst || MODE == kModeFwdLater) && k == P - 1) {
            // (steady: jhi is in range)
            if constexpr (L::FOLD) {
                const uint32_t c = L::cm16(m >> 16);
                cms[jhi] = (uint16_t)(MODE == kModeFwdFirst ? c : max((uint32_t)cm_prev, c));
                if (MODE == kModeFwdFirst || !last_strip) bout[jhi] = (H[R - 1] >> 16) | (f & 0xFFFF0000u);
            } else {
                cms[jhi] = MODE == kModeFwdFirst ? (int)m : max((int)cm_prev, (int)m);
                if (MODE == kModeFwdFirst || !last_strip) bout[jhi] = make_int2((int)H[R - 1], (int)f);
            }
        } else if (REV && k == P - 1) {
            // steady reversed step (16-bit lanes): boundary row out, the stop test
            if constexpr (L::FOLD) {
                if (!last_strip) bout[jhi] = (H[R - 1] >> 16) | (f & 0xFFFF0000u);
                found = (m >> 16) == job.stop_u;
            }
        } else if (MODE == kModeGen && k == P - 1 && (!CHECKED || (jhi >= 0 && jhi < n))) {
            if constexpr (L::FOLD) {
                const uint32_t full = m >> 16;
                if (has_cms) {
                    // the array holds biased u16: merged with the strips above as such
                    if (st == 0) cms[jhi] = (uint16_t)L::cm16(full);
                    else cms[jhi] = (uint16_t)max((uint32_t)cm_prev, L::cm16(full));
                }
                if (!last_strip) bout[jhi] = (H[R - 1] >> 16) | (f & 0xFFFF0000u);
                found = full == job.stop_u;
            } else {
                if (has_cms) {
                    if (st == 0) cms[jhi] = (int)m;
                    else cms[jhi] = max((int)cm_prev, (int)m);
                }
                if (!last_strip) bout[jhi] = make_int2((int)H[R - 1], (int)f);
                found = m == job.stop_u;
            }
        }
        // Reverse fill: stop at the first column where the last strip reaches
        // the target.  Every column up to it is complete in every strip (the
        // earlier strips are ahead), so the first column holding the maximum
        // is at or before it and the strip trackers hold it.
        if ((MODE == kModeGen || REV) && job.stop_u && last_strip && __any_sync(gmask, found)) return true;
        xh = __shfl_sync(gmask, H[R - 1], src);
        xf = __shfl_sync(gmask, f, src);
        xc = __shfl_sync(gmask, m, src);
        return false;
    }

    // Steps [s0, s1) of the current strip: start-up (checked), steady
    // (unchecked), drain (checked).  Returns true on an early stop.  With
    // MAYBE_FAST the steady steps of a one-strip forward fill take the FAST
    // form (the CTA kernel's strips never do).  With MAYBE_MULTI the strips of
    // a forward fill of several strips take the kModeFwdFirst/Later forms;
    // the 8-lane variants (one-strip short reads, whose registers the extra
    // loops would crowd) keep the general step for them.
    template <bool MAYBE_FAST = true, bool MAYBE_MULTI = (P != 8)>
    __device__ bool run(int s0, int s1) {
        const int s_steady = L::FOLD ? 2 * P - 1 : P - 1;
        const int s_drain = max(s_steady, n - 1);
        s1 = min(s1, nsteps);
        int s = s0;
#pragma unroll 1
        for (; s < s1 && s < s_steady; s++)
            if (step<true>(s)) return true;
        const bool fwd = !job.stop_u && has_cms;
        if (MAYBE_FAST && st == 0 && last_strip && fwd && job.ts == 1 && (!L::FOLD || n <= kFastMaxCols)) {
            if constexpr (L::FOLD) {
                // blocks of 4 steps whose max-array values go out in one
                // store (the first steady step's column is 0, so the blocks
                // stay aligned); the last few steady steps run as drain steps
                if ((s - s_steady) % 4 == 0) {
                    const int se = min(s1, s_drain);
                    cpk = ((uint32_t)c_hi << 16) | ((uint32_t)c_lo & 0xFFFFu);
#pragma unroll 1
                    for (; s + 4 <= se; s += 4) {
                        step<false, kModeFast, 0>(s);
                        step<false, kModeFast, 1>(s + 1);
                        step<false, kModeFast, 2>(s + 2);
                        step<false, kModeFast, 3>(s + 3);
                    }
                    c_lo = (int)(int16_t)(cpk & 0xFFFFu);  // (-1: none yet)
                    c_hi = (int)(int16_t)(cpk >> 16);
                }
            } else {
#pragma unroll kUnrollFast
                for (; s < s1 && s < s_drain; s++) step<false, kModeFast>(s);
            }
        } else if (MAYBE_MULTI && fwd && st == 0 && !last_strip && (!L::FOLD || n <= kFastMaxCols)) {
            if constexpr (L::FOLD) cpk = ((uint32_t)c_hi << 16) | ((uint32_t)c_lo & 0xFFFFu);
#pragma unroll kUnrollGen
            for (; s < s1 && s < s_drain; s++) step<false, kModeFwdFirst>(s);
            if constexpr (L::FOLD) {
                c_lo = (int)(int16_t)(cpk & 0xFFFFu);
                c_hi = (int)(int16_t)(cpk >> 16);
            }
        } else if (MAYBE_MULTI && L::FOLD && job.stop_u && n <= kFastMaxCols) {
            // steady reversed steps: no max array, the tracker's columns packed
            if constexpr (L::FOLD) {
                cpk = ((uint32_t)c_hi << 16) | ((uint32_t)c_lo & 0xFFFFu);
                bool stop = false;
#pragma unroll kUnrollGen
                for (; s < s1 && s < s_drain; s++)
                    if (step<false, kModeRev>(s)) {
                        stop = true;
                        break;
                    }
                c_lo = (int)(int16_t)(cpk & 0xFFFFu);
                c_hi = (int)(int16_t)(cpk >> 16);
                if (stop) return true;
            }
        } else if (MAYBE_MULTI && fwd && st > 0 && (!L::FOLD || n <= kFastMaxCols)) {
            if constexpr (L::FOLD) cpk = ((uint32_t)c_hi << 16) | ((uint32_t)c_lo & 0xFFFFu);
#pragma unroll kUnrollGen
            for (; s < s1 && s < s_drain; s++) step<false, kModeFwdLater>(s);
            if constexpr (L::FOLD) {
                c_lo = (int)(int16_t)(cpk & 0xFFFFu);
                c_hi = (int)(int16_t)(cpk >> 16);
            }
        } else {
#pragma unroll kUnrollGen
            for (; s < s1 && s < s_drain; s++)
                if (step<false>(s)) return true;
        }
#pragma unroll 1
        for (; s < s1; s++)
            if (step<true>(s)) return true;
        return false;
    }

    // Strip epilogue: the strip's maximum, its first column, and the first row
    // (within the strip) of that column holding it; the same on every lane.
    __device__ void end(int *v_out, int *c_out, int *row_out) {
        const uint32_t bl = __shfl_sync(gmask, best, gbase + P - 1);
        const int cl = __shfl_sync(gmask, L::FOLD ? c_hi : c_lo, gbase + P - 1);
        const int vfull = lane_hi<L>(bl);
        int cand = INT_MAX;
        if (vfull > 0) {
            if (lane_lo<L>(best) == vfull && c_lo == cl) {
#pragma unroll
                for (int r = R - 1; r >= 0; r--)
                    if (lane_lo<L>(SV[r]) == vfull) cand = k * R + r;
            } else if (L::FOLD && lane_hi<L>(best) == vfull && c_hi == cl) {
#pragma unroll
                for (int r = R - 1; r >= 0; r--)
                    if (lane_hi<L>(SV[r]) == vfull) cand = S + k * R + r;
            }
        }
#pragma unroll
        for (int d = 1; d < P; d <<= 1) cand = min(cand, __shfl_xor_sync(gmask, cand, d));
        *v_out = vfull;
        *c_out = cl;
        *row_out = cand;
        __syncwarp(gmask);
    }
};

// Lexicographic best over strips: larger score, then smaller column, then
// smaller row.
__device__ __forceinline__ void best_merge(int v, int c, int row, int *bv, int *bc, int *br) {
    if (v > *bv || (v == *bv && v > 0 && (c < *bc || (c == *bc && row < *br)))) {
        *bv = v;
        *bc = c;
        *br = row;
    }
}

// The ring fill of one pair by the P lanes of a group, strip after strip.
// All lanes of the group call it with the same job and return the same result.
template <int P, int R, class L, bool DNA>
__device__ RingResult ring_fill(const Job &job, const Scoring &sc, uint32_t *psm, int k, unsigned gmask,
                                int gbase, int lane) {
    using SR = StripRunner<P, R, L, DNA>;
    const int n = job.ncols;
    const int nstrips = (job.mrows + SR::SP - 1) / SR::SP;
    const int pad_top = nstrips * SR::SP - job.mrows;
    typename L::bnd_t *bnd = reinterpret_cast<typename L::bnd_t *>(job.bnd);
    SR sr;
    sr.init(job, sc, psm, k, gmask, gbase, lane, pad_top);
    int g_score = 0, g_col = INT_MAX, g_row = INT_MAX;
#pragma unroll 1
    for (int st = 0; st < nstrips; st++) {
        sr.begin(sc, st, bnd + (size_t)((st + 1) & 1) * n, bnd + (size_t)(st & 1) * n, st == nstrips - 1);
        sr.run(0, sr.nsteps);
        int v, c, row;
        sr.end(&v, &c, &row);
        best_merge(v, c, st * SR::SP + row, &g_score, &g_col, &g_row);
    }
    RingResult res{0, -1, -1, pad_top};
    res.score = g_score;
    res.col = g_score > 0 ? g_col : -1;
    res.row = g_score > 0 ? g_row : -1;
    return res;
}

// Secondary score (item (2)): largest max-array value outside the window
// [end - L, end + L], first column holding it; and the optional max-array
// output.  Reads the column maxima the fill left in the slot scratch.
template <int P, class L>
__device__ void secondary(const BatchView &b, int pair, const Job &job, int end_t, int m, int k, unsigned gmask,
                          int *score2, int *end2) {
    const typename L::cm_t *cms = reinterpret_cast<const typename L::cm_t *>(job.cms);
    const int n = job.ncols;
    const int Lm = b.mask_len >= 0 ? b.mask_len : max(m / 2, 15);
    const long long lo = (long long)end_t - Lm, hi = (long long)end_t + Lm;
    int bv = 0, bj = INT_MAX;
    int32_t *out = (b.flags & GSW_COLMAX) ? b.colmax + b.colmax_off[pair] : nullptr;
    for (int j = k; j < n; j += P) {
        int v;
        if constexpr (L::FOLD) v = (int)cms[j] - 0x8000;
        else v = cms[j];
        if (out) out[j] = v;
        if (end_t >= 0 && j >= lo && j <= hi) continue;
        if (v > bv) { bv = v; bj = j; }
    }
#pragma unroll
    for (int d = 1; d < P; d <<= 1) {
        int ov = __shfl_xor_sync(gmask, bv, d);
        int oj = __shfl_xor_sync(gmask, bj, d);
        if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
    }
    *score2 = bv;
    *end2 = bv > 0 ? bj : -1;
}

// Job of a reverse fill: the query reversed from the end row, the target
// reversed from the end column over the window that must hold the begin.
__device__ __forceinline__ void reverse_job(const BatchView &b, const Scoring &sc, int pair, Job *job) {
    const gsw_result *rp = b.res + pair;
    const int eq = rp->read_end1, et = rp->ref_end1;
    job->q = b.q + b.q_off[pair] + eq;
    job->qs = -1;
    job->mrows = eq + 1;
    job->t = b.t + b.t_off[pair] + et;
    job->ts = -1;
    job->ncols = reverse_window(eq, et, rp->score1, sc);
    job->cms = nullptr;
}

__device__ __forceinline__ void forward_job(const BatchView &b, int pair, Job *job) {
    job->q = b.q + b.q_off[pair];
    job->qs = 1;
    job->mrows = b.q_len[pair];
    job->t = b.t + b.t_off[pair];
    job->ts = 1;
    job->ncols = b.t_len[pair];
    job->stop_u = 0;
}

// Begins from the reversed maximum (one lane writes).
__device__ __forceinline__ void finish_reverse(gsw_result *rp, const RingResult &rr) {
    const int s1 = rp->score1, eq = rp->read_end1, et = rp->ref_end1;
    if (rr.score == s1 && rr.col >= 0) {
        rp->ref_begin1 = et - rr.col;
        rp->read_begin1 = eq - (rr.row - rr.pad_top);
    } else {
        rp->flags |= kResInternal;  // reversed maximum differs from score1
    }
}

// Forward result: score1, ends, secondary score (all P lanes of the group
// call it; the column maxima are in job.cms).
template <int P, class L>
__device__ __forceinline__ void finish_forward(const BatchView &b, const Scoring &sc, int pair, const Job &job,
                                               const RingResult &rr, int k, unsigned gmask) {
    gsw_result *rp = b.res + pair;
    const int m = job.mrows;
    const bool overflow = L::FOLD && rr.score > 32767 - sc.wmax;
    int s2 = 0, e2 = -1;
    const int end_t = rr.col, end_q = rr.score > 0 ? rr.row - rr.pad_top : -1;
    if (!overflow) {
        __syncwarp(gmask);
        secondary<P, L>(b, pair, job, end_t, m, k, gmask, &s2, &e2);
    }
    if (k == 0) {
        rp->score1 = rr.score;
        rp->score2 = s2;
        rp->ref_end1 = end_t;
        rp->read_end1 = end_q;
        rp->ref_begin1 = -1;
        rp->read_begin1 = -1;
        rp->ref_end2 = e2;
        rp->cigar_len = 0;
        rp->cigar_off = -1;
        rp->flags = overflow ? (GSW_RES_S32 | kResPendingS32) : (L::FOLD ? 0 : GSW_RES_S32);
        rp->reserved = 0;
    }
}

// Per-slot scratch of a fill launch: one stride for every variant, so slots
// never overlap when 16-bit and 32-bit tasks run in the same launch.
__device__ __forceinline__ void slot_scratch(const FillScratch &scr, int slot, Job *job) {
    const size_t ncap = (size_t)scr.ncap;
    job->cms = (char *)scr.colmax + slot * ncap * sizeof(int32_t);
    job->bnd = (char *)scr.boundary + slot * 2 * ncap * sizeof(int2);
}

template <int P, int R, class L, bool DNA>
__device__ void run_task(const FillLaunch &fl, int first, int last, uint32_t *wsm, int lane, int slot_base) {
    const int g = lane / P, k = lane % P, gbase = g * P;
    const unsigned gmask = (P == 32) ? 0xFFFFFFFFu : (((1u << P) - 1u) << gbase);
    const int idx = first + g;
    if (idx >= last) return;
    const BatchView &b = fl.b;
    const Scoring &sc = fl.sc;
    const int pair = fl.plan.order[idx];
    gsw_result *rp = b.res + pair;
    uint32_t *psm = wsm;  // the warp's profile region (lane-interleaved)
    if (*fl.bad_letters) {
        // a letter outside the alphabet somewhere in the batch: no letter
        // is read (the steady steps index the profile unclamped)
        if (k == 0 && fl.mode != kFillReverse) {
            rp->score1 = 0; rp->score2 = 0; rp->ref_begin1 = -1; rp->ref_end1 = -1;
            rp->read_begin1 = -1; rp->read_end1 = -1; rp->ref_end2 = -1; rp->cigar_len = 0;
            rp->cigar_off = -1; rp->flags = 0; rp->reserved = 0;
        }
        return;
    }
    Job job;
    slot_scratch(fl.scr, slot_base + g, &job);
    if (fl.mode == kFillReverse) {
        reverse_job(b, sc, pair, &job);
        job.stop_u = L::lane1(rp->score1);
        RingResult rr = ring_fill<P, R, L, DNA>(job, sc, psm, k, gmask, gbase, lane);
        if (k == 0) finish_reverse(rp, rr);
        return;
    }
    // forward (16-bit first pass, or 32-bit rerun)
    const int m = b.q_len[pair], n = b.t_len[pair];
    if (m <= 0 || n <= 0) {
        if (k == 0) {
            rp->score1 = 0; rp->score2 = 0; rp->ref_begin1 = -1; rp->ref_end1 = -1;
            rp->read_begin1 = -1; rp->read_end1 = -1; rp->ref_end2 = -1; rp->cigar_len = 0;
            rp->cigar_off = -1; rp->flags = L::FOLD ? 0 : GSW_RES_S32; rp->reserved = 0;
        }
        if ((b.flags & GSW_COLMAX) && n > 0)
            for (int j = k; j < n; j += P) b.colmax[b.colmax_off[pair] + j] = 0;
        return;
    }
    forward_job(b, pair, &job);
    RingResult rr = ring_fill<P, R, L, DNA>(job, sc, psm, k, gmask, gbase, lane);
    finish_forward<P, L>(b, sc, pair, job, rr, k, gmask);
}

template <int VID>
struct VarC;
#define GSW_VARC(id, P_, R_, S32_)              \
    template <>                                 \
    struct VarC<id> {                           \
        static constexpr int P = P_, R = R_;    \
        using Lanes = std::conditional_t<S32_ != 0, L32, L16>; \
    };
GSW_FILL_VARIANTS(GSW_VARC)
#undef GSW_VARC

// Persistent fill kernel of one variant: warps take tasks (32/P pairs) from
// the variant's counter; the plan sorted them by cost, descending.
// Blocks per SM the compiler keeps each variant's registers for (0: its own
// choice).  Measured on the short-read workload: the 8-lane variants of up
// to 14 row words run best capped at 128 registers (4 blocks of 4 warps);
// the 16-word one keeps its own choice (about 160 registers, 3 blocks).
__host__ __device__ constexpr int fill_min_blocks(int v) {
    return v >= kVarP8First && v < kNumVariants - 1 ? 4 : 0;
}
template <bool DNA, int VID>
__global__ void __launch_bounds__(kBlock, fill_min_blocks(VID)) k_fill(FillLaunch fl, int warp_words) {
    using V = VarC<VID>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (kBlock / 32) + warp;
    uint32_t *wsm = smem + (size_t)warp * warp_words;
    const int slot_base = gwarp * (32 / V::P);
    const int ntasks = fl.plan.task_hi[VID] - fl.plan.task_lo[VID];
    const int first0 = fl.plan.var_start[VID], last = fl.plan.var_start[VID + 1];
    constexpr int per = 32 / V::P;
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&fl.plan.head[VID], 1);
        task = __shfl_sync(0xFFFFFFFFu, task, 0);
        if (task >= ntasks) break;
        run_task<V::P, V::R, typename V::Lanes, DNA>(fl, first0 + task * per, last, wsm, lane, slot_base);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// CTA kernel for pairs whose query spans many strips.  Strip x reads only the
// bottom row (H, F) and the running column maxima that strip x-1 leaves in
// global scratch, one column at a time, so several strips of a pair can run
// at once when each stays far enough behind the one above it.  The warps of
// the CTA (one 32-lane folded ring each; in 16-bit lanes 1,024 rows per strip
// for DNA, 512 for general alphabets) advance in phases of kLongChunk steps
// separated by a CTA barrier, which
// also makes the previous phases' global writes visible.  Strip x+1 starts
// long_lag() phases after strip x, so every boundary word and column maximum
// it reads (one block of 32 columns ahead) was written in a completed phase,
// and the ping-pong boundary buffer it writes was read a phase earlier.
//
// One thread schedules between the two barriers of a phase: it merges the
// results of strips that ended, hands a finished pair to one warp (secondary
// score or begins), hands strips to idle warps (oldest pair first, the next
// strip of a pair no earlier than long_lag() phases after the previous one),
// and opens the next pair of the class in a free scratch slot, so the end of
// one pair overlaps the start of the next.
constexpr int kLongChunk = 128;
constexpr int kLongSlots = 4;  // pairs in flight per CTA

template <class L>
__host__ __device__ constexpr int long_lag() {
    // strip x-1 writes column j at its step j + dw; strip x reads columns up
    // to s + 2P - 1 at step s: (lag - 1) * C >= 2P - 1 + dw
    constexpr int P = 32, dw = L::FOLD ? 2 * P - 1 : P - 1;
    return 1 + (2 * P - 1 + dw + kLongChunk - 1) / kLongChunk;
}

// Lag of a banded reversed fill, whose strip x+1 starts up to SP columns
// right of strip x: strip x+1 reads absolute column c0(x+1) + s + 2P - 1 at
// its step s, which strip x writes at its step c0(x+1) - c0(x) + s + 2P - 1
// + dw, so (lag - 1) * C >= SP + 2P - 1 + dw (16-bit DNA lanes: 10 phases).  The
// same lag keeps strip x+2's writes after strip x+1's reads of the ping-pong
// buffer (lag * C + dw > SP).
template <class L, int SP>
__host__ __device__ constexpr int long_lag_band() {
    constexpr int P = 32, dw = L::FOLD ? 2 * P - 1 : P - 1;
    return 1 + (SP + 2 * P - 1 + dw + kLongChunk - 1) / kLongChunk;
}

struct LongSlot {
    Job job;
    int pair;  // -1: free
    int seq;   // order in which the pairs were opened
    int nstrips, pad_top;
    int next;        // next strip to hand out
    int last_start;  // phase at which the last handed-out strip started
    int running;     // strips running
    int stopped;     // the last strip found the reverse target
    int fin;         // finalisation handed out
    int bv, bc, br;  // merged maximum, its column and (padded) row
    int band;        // reversed fill restricted to the reverse band (below)
    int G, Gn;       // reverse band [-Gn, G] around the main diagonal
    int lag;         // phases between the starts of consecutive strips
};

// Columns [c0, c1] of strip x of a banded reversed fill: every path reaching
// score1 starts at the reversed origin and keeps j - i within [-Gn, G] (the
// band kernel's argument), so the strip's rows [r0, r1] need only the
// columns [r0 - Gn, r1 + G] of the window, plus the column left of them: the
// first row's band cell (r0, r0 - Gn) takes its diagonal predecessor from the
// boundary row at column r0 - Gn - 1, and the strip reads its boundary row
// one column behind the cell it computes.  Cells outside the band are never
// on such a path; what a strip reads from outside its neighbour's columns
// (the top boundary right of the strip above) is H = 0 and F = -inf, a lower
// bound like any restriction of the local DP, so the band's values on those
// paths are the full DP's.  c1 < c0: the band misses the window.
__device__ __forceinline__ void band_cols(const LongSlot &S, int strip, int SP, int *c0, int *c1) {
    if (!S.band) {
        *c0 = 0;
        *c1 = S.job.ncols - 1;
        return;
    }
    const int r0 = max(0, strip * SP - S.pad_top), r1 = (strip + 1) * SP - 1 - S.pad_top;
    *c0 = max(0, r0 - S.Gn - 1);
    *c1 = min(S.job.ncols - 1, r1 + S.G);
}

struct LongCmd {
    int slot;   // -1: idle
    int strip;  // >= 0: strip to run; -1: finalise the slot's pair
    int start;  // phase at which the strip started
};

struct LongRep {
    int ended;  // the strip ended (or the finalisation finished) this phase
    int v, c, row, stop;
};

template <int NW>
struct LongShared {
    LongSlot slot[kLongSlots];
    LongCmd cmd[NW];
    LongRep rep[NW];
    int seq, exhausted, done;
};

// Opens the next pair of class CLS in slot s; false when none is left.
template <class L, int SP>
__device__ bool long_open(const FillLaunch &fl, int cls, LongSlot &S, int s, int seq) {
    const int ntasks = fl.plan.task_hi[cls] - fl.plan.task_lo[cls];
    const int t = atomicAdd(&fl.plan.head[cls], 1);
    if (t >= ntasks) return false;
    const int pair = fl.plan.order[fl.plan.var_start[cls] + t];
    Job job;
    slot_scratch(fl.scr, blockIdx.x * kLongSlots + s, &job);
    S.band = 0;
    S.G = S.Gn = 0;
    if (fl.mode == kFillReverse) {
        reverse_job(fl.b, fl.sc, pair, &job);
        const gsw_result r = fl.b.res[pair];
        job.stop_u = L::lane1(r.score1);
        // the band pays when it takes at least a quarter off every strip
        const int G = reverse_gap_bound(r.read_end1, r.score1, fl.sc);
        const int Gn = reverse_gap_bound_rows(r.read_end1, r.score1, fl.sc);
        if (G >= 0 && ((long long)SP + G + Gn + 1) * 4 <= 3LL * job.ncols) {
            S.band = 1;
            S.G = G;
            S.Gn = Gn;
        }
    } else {
        forward_job(fl.b, pair, &job);
    }
    S.lag = S.band ? long_lag_band<L, SP>() : long_lag<L>();
    S.job = job;
    S.pair = pair;
    S.seq = seq;
    S.nstrips = (job.mrows + SP - 1) / SP;
    S.pad_top = S.nstrips * SP - job.mrows;
    S.next = 0;
    S.last_start = 0;
    S.running = 0;
    S.stopped = 0;
    S.fin = 0;
    S.bv = 0;
    S.bc = INT_MAX;
    S.br = INT_MAX;
    return true;
}

template <class L, int NW, int SP>
__device__ void long_schedule(const FillLaunch &fl, int cls, LongShared<NW> &sh, int ph) {
    // results of strips that ended, finished finalisations
    for (int w = 0; w < NW; w++) {
        if (!sh.rep[w].ended) continue;
        sh.rep[w].ended = 0;
        LongCmd &c = sh.cmd[w];
        LongSlot &S = sh.slot[c.slot];
        if (c.strip < 0) {
            S.pair = -1;
        } else {
            best_merge(sh.rep[w].v, sh.rep[w].c, sh.rep[w].row, &S.bv, &S.bc, &S.br);
            S.running--;
            if (sh.rep[w].stop) S.stopped = 1;
        }
        c.slot = -1;
    }
    // idle warps: finalisations first, then strips of the oldest pair that
    // may start one, then a new pair
    for (int w = 0; w < NW; w++) {
        LongCmd &c = sh.cmd[w];
        if (c.slot >= 0) continue;
        int pick = -1;
        for (int s = 0; s < kLongSlots; s++) {
            const LongSlot &S = sh.slot[s];
            if (S.pair >= 0 && !S.fin && S.running == 0 && (S.stopped || S.next == S.nstrips)) {
                pick = s;
                break;
            }
        }
        if (pick >= 0) {
            sh.slot[pick].fin = 1;
            c.slot = pick;
            c.strip = -1;
            c.start = ph;
            continue;
        }
        int best_seq = INT_MAX;
        for (int s = 0; s < kLongSlots; s++) {
            const LongSlot &S = sh.slot[s];
            if (S.pair >= 0 && !S.stopped && S.next < S.nstrips && (S.next == 0 || ph >= S.last_start + S.lag) &&
                S.seq < best_seq) {
                best_seq = S.seq;
                pick = s;
            }
        }
        if (pick < 0 && !sh.exhausted) {
            for (int s = 0; s < kLongSlots; s++) {
                if (sh.slot[s].pair >= 0) continue;
                if (long_open<L, SP>(fl, cls, sh.slot[s], s, sh.seq)) {
                    sh.seq++;
                    pick = s;
                } else {
                    sh.exhausted = 1;
                }
                break;
            }
        }
        if (pick < 0) break;  // nothing can start in this phase
        LongSlot &S = sh.slot[pick];
        c.slot = pick;
        c.strip = S.next++;
        c.start = ph;
        S.last_start = ph;
        S.running++;
    }
    bool busy = !sh.exhausted;
    for (int s = 0; s < kLongSlots; s++) busy |= sh.slot[s].pair >= 0;
    sh.done = busy ? 0 : 1;
}

template <bool DNA, bool S32>
struct LongCfg {
    using L = std::conditional_t<S32, L32, L16>;
    // DNA in 16-bit lanes: 16 row words per lane (1,024 rows per strip), so
    // the per-step work of a lane (letters, profile loads, shuffles, tracker
    // bookkeeping, boundary and max-array traffic) is spread over 32 cells;
    // 4 warps per CTA and 3 CTAs per SM (168 registers a thread, 64 KB of
    // profile per CTA).  Measured on 10,000 long reads against 8 row words and
    // 8 warps (2 CTAs per SM): forward fill 265 -> 218 ms, reverse 105 -> 91
    // ms; 12 or 20-24 row words, 2 or 8 warps per CTA were slower.
    static constexpr int P = 32, R = (DNA && !S32) ? 16 : 8;
    static constexpr int NW = 4;
    static constexpr int MINB = DNA ? 3 : 4;
    static constexpr int SP = S32 ? P * R : 2 * P * R;
    static constexpr int CLS = S32 ? kClassLong32 : kClassLong16;
};

template <bool DNA, bool S32>
__global__ void __launch_bounds__(LongCfg<DNA, S32>::NW * 32, LongCfg<DNA, S32>::MINB)
    k_fill_long(FillLaunch fl, int warp_words) {
    using C = LongCfg<DNA, S32>;
    using L = typename C::L;
    constexpr int NW = C::NW, SP = C::SP;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ LongShared<NW> sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *psm = smem + (size_t)warp * warp_words;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kLongSlots; s++) sh.slot[s].pair = -1;
        for (int w = 0; w < NW; w++) {
            sh.cmd[w].slot = -1;
            sh.rep[w].ended = 0;
        }
        sh.seq = 0;
        sh.exhausted = 0;
        sh.done = 0;
    }
    StripRunner<C::P, C::R, L, DNA> sr;
    int strip_c0 = 0;  // first window column of the warp's strip
#pragma unroll 1
    for (int ph = 0;; ph++) {
        __syncthreads();
        if (threadIdx.x == 0) long_schedule<L, NW, SP>(fl, C::CLS, sh, ph);
        __syncthreads();
        if (sh.done) break;
        const LongCmd cmd = sh.cmd[warp];
        if (cmd.slot < 0) continue;
        const LongSlot &S = sh.slot[cmd.slot];
        if (cmd.strip < 0) {
            RingResult rr;
            rr.score = S.bv;
            rr.col = S.bv > 0 ? S.bc : -1;
            rr.row = S.bv > 0 ? S.br : -1;
            rr.pad_top = S.pad_top;
            if (fl.mode == kFillReverse) {
                if (lane == 0) finish_reverse(fl.b.res + S.pair, rr);
            } else {
                finish_forward<32, L>(fl.b, fl.sc, S.pair, S.job, rr, lane, 0xFFFFFFFFu);
            }
            if (lane == 0) sh.rep[warp].ended = 1;
            continue;
        }
        if (ph == cmd.start) {
            using bnd_t = typename L::bnd_t;
            bnd_t *bnd = reinterpret_cast<bnd_t *>(S.job.bnd);
            const size_t n = (size_t)S.job.ncols;
            // the strip's columns (all of the window unless banded): its
            // letters, boundary reads and writes start at column c0
            int c1;
            band_cols(S, cmd.strip, SP, &strip_c0, &c1);
            Job jb = S.job;
            jb.t = S.job.t + (long long)strip_c0 * S.job.ts;
            jb.ncols = max(0, c1 - strip_c0 + 1);
            bnd_t *bout = bnd + (cmd.strip & 1) * n;
            if (S.band && cmd.strip + 1 < S.nstrips) {
                // the next strip's columns right of this strip's last one
                // read the outside value: H = 0, F = -inf (biased -O)
                int n0, n1;
                band_cols(S, cmd.strip + 1, SP, &n0, &n1);
                bnd_t out;
                if constexpr (L::FOLD) out = L::lane1(0) | (L::lane1(-fl.sc.O) << 16);
                else out = make_int2(0, -fl.sc.O);
                for (int c = max(n0, jb.ncols > 0 ? c1 + 1 : n0) + lane; c <= n1; c += 32) bout[c] = out;
            }
            sr.init(jb, fl.sc, psm, lane, 0xFFFFFFFFu, 0, lane, S.pad_top);
            sr.begin(fl.sc, cmd.strip, bnd + ((cmd.strip + 1) & 1) * n + strip_c0, bout + strip_c0,
                     cmd.strip == S.nstrips - 1);
        }
        bool stop = false, fin = S.stopped != 0;
        if (!fin) {
            const int q = ph - cmd.start;
            stop = sr.template run<false>(q * kLongChunk, (q + 1) * kLongChunk);
            fin = stop || (q + 1) * kLongChunk >= sr.nsteps;
        }
        if (fin) {
            int v, c, row;
            sr.end(&v, &c, &row);
            if (lane == 0) {
                LongRep &r = sh.rep[warp];
                r.v = v;
                r.c = v > 0 ? c + strip_c0 : c;  // the window's column
                r.row = cmd.strip * SP + row;
                r.stop = stop ? 1 : 0;
                r.ended = 1;
            }
        }
    }
}

template <bool DNA, bool S32>
size_t long_smem_bytes(int A) {
    using C = LongCfg<DNA, S32>;
    return (size_t)prof_words(C::R, C::L::FOLD, DNA, A) * 32 * sizeof(uint32_t) * C::NW;
}

template <bool DNA, bool S32>
int long_occupancy(int A) {
    using C = LongCfg<DNA, S32>;
    const size_t sm = long_smem_bytes<DNA, S32>(A);
    cudaFuncSetAttribute(k_fill_long<DNA, S32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill_long<DNA, S32>, C::NW * 32, sm);
    return nb;
}

template <bool DNA, bool S32>
cudaError_t launch_long(const FillLaunch &fl, int sms, int max_blocks, cudaStream_t st) {
    using C = LongCfg<DNA, S32>;
    if (!((fl.class_mask >> C::CLS) & 1u)) return cudaSuccess;  // no pair of the class
    const size_t sm = long_smem_bytes<DNA, S32>(fl.sc.A);
    const int nb = long_occupancy<DNA, S32>(fl.sc.A);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * nb;
    grid = std::min(grid, max_blocks);
    grid = std::min(grid, fl.scr.nslots / kLongSlots);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    k_fill_long<DNA, S32><<<grid, C::NW * 32, sm, st>>>(fl, (int)(sm / sizeof(uint32_t) / C::NW));
    return cudaGetLastError();
}

template <bool DNA, int VID>
size_t smem_bytes(int A) {
    using V = VarC<VID>;
    return (size_t)prof_words(V::R, V::Lanes::FOLD, DNA, A) * 32 * sizeof(uint32_t) * (kBlock / 32);
}

template <bool DNA, int VID>
int occupancy(int A) {
    const size_t sm = smem_bytes<DNA, VID>(A);
    cudaFuncSetAttribute(k_fill<DNA, VID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill<DNA, VID>, kBlock, sm);
    return nb;
}

template <bool DNA, int VID>
cudaError_t launch_one(const FillLaunch &fl, int sms, int max_blocks, cudaStream_t st) {
    if (!((fl.class_mask >> VID) & 1u)) return cudaSuccess;  // no pair of the class
    const size_t sm = smem_bytes<DNA, VID>(fl.sc.A);
    int nb = occupancy<DNA, VID>(fl.sc.A);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * nb;
    if (grid > max_blocks) grid = max_blocks;
    // every pair in flight has a slot: never more warps than the slots hold
    grid = std::min(grid, fl.scr.nslots / ((kBlock / 32) * (32 / VarC<VID>::P)));
    if (grid < 1) return cudaErrorInvalidConfiguration;
    k_fill<DNA, VID><<<grid, kBlock, sm, st>>>(fl, (int)(sm / sizeof(uint32_t) / (kBlock / 32)));
    return cudaGetLastError();
}

template <bool DNA>
cudaError_t launch_all(const FillLaunch &fl, int sms, int max_blocks, cudaStream_t st) {
    // heaviest classes first: the CTA kernel for queries of many strips, then
    // the per-group variants by rows per strip
    cudaError_t e = launch_long<DNA, true>(fl, sms, max_blocks, st);
    if (e == cudaSuccess) e = launch_long<DNA, false>(fl, sms, max_blocks, st);
#define GSW_LAUNCH(id, P_, R_, S_) \
    if (e == cudaSuccess) e = launch_one<DNA, kNumVariants - 1 - id>(fl, sms, max_blocks, st);
    GSW_FILL_VARIANTS(GSW_LAUNCH)
#undef GSW_LAUNCH
    return e;
}

template <bool DNA>
int max_slots(int A, int sms) {
    int best = 0;
#define GSW_SLOTS(id, P_, R_, S_)                                                   \
    {                                                                             \
        const int nb = occupancy<DNA, id>(A);                                     \
        const int slots = sms * nb * (kBlock / 32) * (32 / VarC<id>::P);          \
        best = slots > best ? slots : best;                                       \
    }
    GSW_FILL_VARIANTS(GSW_SLOTS)
#undef GSW_SLOTS
    return best;
}

}  // namespace

int fill_block_threads() { return kBlock; }

int fill_max_pairs_per_warp() {
    int most = 1;
#define GSW_PER_WARP(id, P_, R_, S_) most = 32 / P_ > most ? 32 / P_ : most;
    GSW_FILL_VARIANTS(GSW_PER_WARP)
#undef GSW_PER_WARP
    return most;
}

// Slots (pairs in flight) the largest variant launch can hold, at full
// occupancy on `sms` SMs; a launch is never given more blocks than
// max_blocks, so callers can cap the scratch.
int fill_slots(const Scoring &sc, int sms) { return sc.dna4 ? max_slots<true>(sc.A, sms) : max_slots<false>(sc.A, sms); }

cudaError_t launch_fill(const FillLaunch &fl, int sms, int max_blocks, cudaStream_t st) {
    return fl.sc.dna4 ? launch_all<true>(fl, sms, max_blocks, st) : launch_all<false>(fl, sms, max_blocks, st);
}


// ---------------------------------------------------------------------------
// Allocation-free forward fill (gsw_fill_static).  Its per-slot scratch (the
// column maxima and strip boundaries of a pair in flight) lives in a
// file-scope device array instead of context memory.
namespace {

constexpr int kStaticMaxTarget = GSW_STATIC_MAX_TARGET;
constexpr size_t kStaticSlotBytes = (size_t)kStaticMaxTarget * sizeof(int32_t) + 2 * (size_t)kStaticMaxTarget * sizeof(int2);
static_assert(kStaticMaxTarget % 4 == 0 && kStaticSlotBytes % 16 == 0,
              "slots start on 16-byte boundaries (the fill's 8-byte max-array stores)");
constexpr int kStaticWarps = 152 * 4;                 // warps of one launch
constexpr int kStaticSlots = kStaticWarps * 2;        // two pairs in flight per warp
constexpr size_t kStaticErrOff = kStaticSlotBytes * kStaticSlots;
constexpr size_t kStaticBytes = kStaticErrOff + 256;  // + the per-call error word
static_assert(kStaticBytes == GSW_STATIC_SCRATCH_BYTES, "header states the scratch size");

static __device__ __align__(256) uint8_t g_static_scratch[kStaticBytes];

template <int R, class L, bool DNA>
__device__ bool static_fill_pair(const BatchView &b, const Scoring &sc, int pair, uint32_t *wsm, int lane, int k,
                                 unsigned gmask, int gbase, uint8_t *slot) {
    gsw_result *rp = b.res + pair;
    Job job;
    job.q = b.q + b.q_off[pair];
    job.qs = 1;
    job.mrows = b.q_len[pair];
    job.t = b.t + b.t_off[pair];
    job.ts = 1;
    job.ncols = b.t_len[pair];
    job.stop_u = 0;
    job.cms = slot;
    job.bnd = slot + (size_t)kStaticMaxTarget * sizeof(int32_t);
    const RingResult rr = ring_fill<16, R, L, DNA>(job, sc, wsm, k, gmask, gbase, lane);
    if (L::FOLD && rr.score > 32767 - sc.wmax) return false;  // refill in 32-bit lanes
    int s2 = 0, e2 = -1;
    const int end_t = rr.col, end_q = rr.score > 0 ? rr.row - rr.pad_top : -1;
    __syncwarp(gmask);
    secondary<16, L>(b, pair, job, end_t, job.mrows, k, gmask, &s2, &e2);
    if (k == 0) {
        rp->score1 = rr.score;
        rp->score2 = s2;
        rp->ref_end1 = end_t;
        rp->read_end1 = end_q;
        rp->ref_begin1 = -1;
        rp->read_begin1 = -1;
        rp->ref_end2 = e2;
        rp->cigar_len = 0;
        rp->cigar_off = -1;
        rp->flags = L::FOLD ? 0 : GSW_RES_S32;
        rp->reserved = 0;
    }
    return true;
}

// Warps take two pairs at a time (one per 16-lane group), grid-stride.  Both
// groups of a warp use the same row-word count R, because their profiles
// share the warp's interleaved shared-memory region; a group whose 16-bit
// fill overflowed refills afterwards in 32-bit lanes.
template <bool DNA>
__global__ void __launch_bounds__(kBlock) k_fill_static(BatchView b, Scoring sc, uint8_t *scratch, int warp_words) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 4, k = lane & 15, gbase = g * 16;
    const unsigned gmask = 0xFFFFu << gbase;
    const int gwarp = blockIdx.x * (blockDim.x / 32) + warp;
    const int nwarps = gridDim.x * (blockDim.x / 32);
    uint32_t *wsm = smem + (size_t)warp * warp_words;
    uint8_t *slot = scratch + (size_t)(gwarp * 2 + g) * kStaticSlotBytes;
    int32_t *err = reinterpret_cast<int32_t *>(scratch + kStaticErrOff);
    for (int base = gwarp * 2; base < b.npairs; base += nwarps * 2) {
        const int pair = base + g;
        const bool has = pair < b.npairs;
        // the checks gsw_align_batch makes before any fill, made here by
        // each group before its pair's first access: lengths in [0, 2^24),
        // offsets >= 0 and targets within the slot; then the letter codes
        int m = 0, n = 0;
        bool bad = false;
        if (has) {
            m = b.q_len[pair];
            n = b.t_len[pair];
            bad = (uint32_t)m >= (1u << 24) || (uint32_t)n >= (1u << 24) || b.q_off[pair] < 0 || b.t_off[pair] < 0 ||
                  ((b.flags & GSW_COLMAX) && b.colmax_off[pair] < 0) || n > kStaticMaxTarget;
        }
        if (has && !bad) {
            const uint8_t *qp = b.q + b.q_off[pair], *tp = b.t + b.t_off[pair];
            int found = 0;
            for (int i = k; i < m; i += 16) found |= qp[i] >= sc.A;
            for (int j = k; j < n; j += 16) found |= tp[j] >= sc.A;
            bad = __any_sync(gmask, found) != 0;
        }
        const bool empty = has && !bad && (m == 0 || n == 0);
        const bool run = has && !bad && !empty;
        if (has && k == 0 && (bad || empty)) {
            gsw_result *rp = b.res + pair;
            rp->score1 = 0; rp->score2 = 0; rp->ref_begin1 = -1; rp->ref_end1 = -1; rp->read_begin1 = -1;
            rp->read_end1 = -1; rp->ref_end2 = -1; rp->cigar_len = 0; rp->cigar_off = -1;
            rp->flags = bad ? kResInvalid : 0;
            rp->reserved = 0;
            if (bad) atomicOr(err, 1);
        }
        if (empty && (b.flags & GSW_COLMAX))
            for (int j = k; j < n; j += 16) b.colmax[b.colmax_off[pair] + j] = 0;
        const int rows = __reduce_max_sync(0xFFFFFFFFu, run ? m : 0);
        bool ok = true;
        if (run) {
            if (rows <= 64) ok = static_fill_pair<2, L16, DNA>(b, sc, pair, wsm, lane, k, gmask, gbase, slot);
            else if (rows <= 128) ok = static_fill_pair<4, L16, DNA>(b, sc, pair, wsm, lane, k, gmask, gbase, slot);
            else if (rows <= 192) ok = static_fill_pair<6, L16, DNA>(b, sc, pair, wsm, lane, k, gmask, gbase, slot);
            else ok = static_fill_pair<8, L16, DNA>(b, sc, pair, wsm, lane, k, gmask, gbase, slot);
        }
        __syncwarp();
        if (!ok) static_fill_pair<8, L32, DNA>(b, sc, pair, wsm, lane, k, gmask, gbase, slot);
        __syncwarp();
    }
}

struct StaticSetup {
    bool done = false;
    uint8_t *ptr = nullptr;
};
StaticSetup g_static_setup[64];
std::mutex g_static_mu;

}  // namespace

}  // namespace gsw

extern "C" int gsw_fill_static(int32_t npairs, const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                               const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                               int32_t max_target_len, const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                               int32_t gap_extend, uint32_t flags, int32_t mask_len, gsw_result *results,
                               int32_t *colmax, const int64_t *colmax_off, void *stream) {
    using namespace gsw;
    if (npairs < 0) return set_err(GSW_EINVAL, "npairs < 0");
    if (flags & ~(uint32_t)GSW_COLMAX) return set_err(GSW_EINVAL, "flags other than GSW_COLMAX (0x%x)", flags);
    if (max_target_len < 0 || max_target_len > kStaticMaxTarget)
        return set_err(GSW_EINVAL, "max_target_len %d not in [0, %d]", max_target_len, kStaticMaxTarget);
    if (mask_len > (1 << 30)) return set_err(GSW_EINVAL, "mask_len too large");
    Scoring sc;
    {
        const int e = make_scoring(matrix, alphabet, gap_open, gap_extend, &sc);
        if (e != GSW_OK) return e;
    }
    if (npairs == 0) return GSW_OK;
    if (!q || !q_off || !q_len || !t || !t_off || !t_len || !results)
        return set_err(GSW_EINVAL, "NULL input or result pointer");
    if ((flags & GSW_COLMAX) && (!colmax || !colmax_off)) return set_err(GSW_EINVAL, "colmax output missing");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set_err(GSW_ECUDA, "no current device");
    const size_t per_warp = (size_t)prof_words(8, true, sc.dna4 != 0, alphabet) * 32 * sizeof(uint32_t);
    int wpb = (int)((200u << 10) / per_warp);
    wpb = wpb > 4 ? 4 : (wpb < 1 ? 1 : wpb);
    const size_t smem = per_warp * wpb;
    uint8_t *scratch;
    {
        // once per device, with that device current: the device address of
        // the static scratch (the host-side symbol is only a stand-in)
        std::lock_guard<std::mutex> lk(g_static_mu);
        StaticSetup &su = g_static_setup[dev];
        if (!su.done) {
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess) return set_err(GSW_ECUDA, "scratch address: %s", cudaGetErrorString(e));
            if (cudaFuncSetAttribute(k_fill_static<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(k_fill_static<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10) !=
                    cudaSuccess)
                return set_err(GSW_ECUDA, "kernel shared-memory limit");
            su.ptr = static_cast<uint8_t *>(ptr);
            su.done = true;
        }
        scratch = su.ptr;
    }
    BatchView bv;
    memset(&bv, 0, sizeof(bv));
    bv.q = q; bv.q_off = q_off; bv.q_len = q_len;
    bv.t = t; bv.t_off = t_off; bv.t_len = t_len;
    bv.res = results;
    bv.npairs = npairs;
    bv.flags = flags;
    bv.mask_len = mask_len;
    bv.colmax = colmax;
    bv.colmax_off = colmax_off;
    cudaStream_t st = (cudaStream_t)stream;
    // the error word must start at zero; the slots need no clearing
    if (cudaMemsetAsync(scratch + kStaticErrOff, 0, sizeof(int32_t), st) != cudaSuccess)
        return set_err(GSW_ECUDA, "clearing the error word");
    const int grid = kStaticWarps / wpb;
    if (sc.dna4) k_fill_static<true><<<grid, wpb * 32, smem, st>>>(bv, sc, scratch, (int)(per_warp / 4));
    else k_fill_static<false><<<grid, wpb * 32, smem, st>>>(bv, sc, scratch, (int)(per_warp / 4));
    {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_err(GSW_ECUDA, "fill launch: %s", cudaGetErrorString(e));
    }
    int32_t err = 0;
    if (cudaMemcpyAsync(&err, scratch + kStaticErrOff, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_err(GSW_ECUDA, "error-word readback");
    if (err)
        return set_err(GSW_EINVAL, "pairs with a length outside [0, 2^24), a target over %d letters, a negative "
                                   "offset or a letter code >= %d (records flagged GSW_RES_INVALID)",
                       kStaticMaxTarget, alphabet);
    return GSW_OK;
}

namespace gsw {
}  // namespace gsw
