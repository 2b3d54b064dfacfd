// C entry points over the library's host-side geometry rules (gsw_impl.cuh),
// compiled by g++ for the CPU tests of those rules: the reverse fill's window
// and band, the traceback band, the traceback class routing, the fill classes
// and the launch mask, and the status a batch returns from its kernels' counts.
#include "gsw_impl.cuh"

namespace {
gsw::Scoring scoring(int A, const signed char *W, int O, int X) {
    gsw::Scoring sc{};
    sc.A = A;
    sc.O = O;
    sc.X = X;
    int mx = W[0], mn = W[0];
    for (int k = 0; k < A * A; ++k) {
        mx = W[k] > mx ? W[k] : mx;
        mn = W[k] < mn ? W[k] : mn;
        sc.W[k] = W[k];
    }
    sc.wmax = mx;
    sc.wmin = mn;
    sc.dna4 = A == 4;
    return sc;
}
}  // namespace

extern "C" {

// fill class of a pair (mode 0 forward, 2 reverse) under a tune table
// (GSW_TUNE_BUCKETS codes, -1: default rule)
int hr_pick_class(int A, const signed char *W, int O, int X, const signed char *table, int mode, int rows, int s32) {
    gsw::Scoring sc = scoring(A, W, O, X);
    for (int b = 0; b < GSW_TUNE_BUCKETS; ++b) sc.fill_class[b] = table[b];
    return mode == gsw::kFillForward ? gsw::pick_class16(rows, sc) : gsw::pick_class_reverse(rows, s32 != 0, sc);
}

unsigned hr_fill_class_mask(int A, const signed char *W, int O, int X, const signed char *table, int mode, int maxm,
                            int force_s32, int s32) {
    gsw::Scoring sc = scoring(A, W, O, X);
    for (int b = 0; b < GSW_TUNE_BUCKETS; ++b) sc.fill_class[b] = table[b];
    return gsw::fill_class_mask(mode, maxm, sc, force_s32 != 0, s32 != 0);
}

int hr_reverse_window(int A, const signed char *W, int O, int X, int end_q, int end_t, int score1) {
    return gsw::reverse_window(end_q, end_t, score1, scoring(A, W, O, X));
}

int hr_reverse_gap_bound(int A, const signed char *W, int O, int X, int end_q, int score1) {
    return gsw::reverse_gap_bound(end_q, score1, scoring(A, W, O, X));
}

int hr_reverse_gap_bound_rows(int A, const signed char *W, int O, int X, int end_q, int score1) {
    return gsw::reverse_gap_bound_rows(end_q, score1, scoring(A, W, O, X));
}

int hr_band_range(int A, const signed char *W, int O, int X, int la, int lb, int score1, int *dlo, int *dhi) {
    return gsw::band_range(la, lb, score1, scoring(A, W, O, X), dlo, dhi);
}

int hr_trace_class(int A, const signed char *W, int O, int X, int la, int lb, int score1, int small, int *dlo,
                   int *dhi) {
    return gsw::trace_class(la, lb, score1, scoring(A, W, O, X), small != 0, dlo, dhi);
}

long long hr_t16_need_words(int la, int lb, int v) { return gsw::t16_need_words(la, lb, v); }

int hr_batch_status(int bad_letters, unsigned long long internal, int cigar, unsigned long long words,
                    long long capacity) {
    return gsw::batch_status(bad_letters, internal, cigar != 0, words, capacity);
}

}  // extern "C"
