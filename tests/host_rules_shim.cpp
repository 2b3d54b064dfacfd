// C entry points over the library's host-side geometry rules (gsw_impl.cuh),
// compiled by g++ for the CPU tests of those rules: the reverse fill's window
// and band, the traceback band, the traceback class routing, and the status a
// batch returns from its kernels' counts.
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
