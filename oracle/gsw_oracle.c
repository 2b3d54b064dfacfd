/*
 * Oracle for the SSW method (Zhao, Lee, Garrison, Marth 2012, "SSW Library: An
 * SIMD Smith-Waterman C/C++ Library for Use in Genomic Applications").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of what the method computes.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library never
 * links it, and it shares no code, header or table with the CUDA path.
 *
 * Everything is int32 and full-matrix; no blocking, striping, banding or lane
 * packing.  Notation: query q (length m, rows i), target t (length n, columns
 * j), substitution matrix W[a*A + b] = score of query letter a against target
 * letter b, gap open O and gap extend X given as non-negative integers with
 * O >= X, so that a gap of length k costs O + (k-1)*X.
 *
 *   ora_fill        local Smith-Waterman-Gotoh fill (Intro; Algorithm (1)): the
 *                   per-column maximum ("max" array), the optimal score and the
 *                   end cell, found from the max array and from the recorded
 *                   column that holds the matrix maximum.
 *   ora_secondary   suboptimal score from the max array with the primary's
 *                   neighbourhood masked (Algorithm (2); Fig. 1 caption).
 *   ora_begin       reversed SW from the end to find the begin (Algorithm (1);
 *                   Fig. 1 caption, "much smaller, locally computed matrix").
 *   ora_cigar       global Gotoh between begin and end with an explicit
 *                   three-state traceback (Algorithm (1), "the banded SW ...
 *                   generates the detailed alignment"; the oracle fills the
 *                   whole rectangle, no band).
 *   ora_align       the four steps for one pair; ora_align_batch over a batch
 *                   with one pthread per core.
 *
 * Readings of the paper (it prints no equations):
 *   - H(i,j) = max(0, H(i-1,j-1) + W(q_i,t_j), E(i,j), F(i,j)),
 *     E(i,j) = max(H(i,j-1) - O, E(i,j-1) - X), F(i,j) = max(H(i-1,j) - O,
 *     F(i-1,j) - X); H = 0 and E = F = -inf before the first row and column.
 *   - End: the first column (smallest j) whose max equals the matrix maximum,
 *     then the first row (smallest i) in that column with that value: the
 *     column is recorded only when the maximum strictly improves.
 *   - Secondary: the mask is the window [end_t - L, end_t + L] of the max
 *     array, L = mask_len (default max(m/2, 15)); score2 is the largest
 *     unmasked entry and ref_end2 its first column; score2 = 0 gives -1.
 *   - Begin: the local fill on reverse(q[0..end_q]) x reverse(t[0..end_t]) with
 *     the same end rule; begin = end - (reversed end).  Every optimal alignment
 *     inside that prefix rectangle ends exactly at the end cell, so this picks
 *     the optimal alignment ending there with the largest begin on the target,
 *     then the largest begin on the query.
 *   - CIGAR: from (end_q, end_t) in state H; in H prefer the diagonal (M) if
 *     H == H(i-1,j-1) + W, else the horizontal gap state E (D, consumes target)
 *     if H == E, else the vertical gap state F (I, consumes query); in E take
 *     the open (back to H at j-1) if E == H(i,j-1) - O, else extend; the same
 *     in F.  Runs are encoded (len << 4) | op with M = 0, I = 1, D = 2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORA_NEG (-(1 << 30))

#define ORA_OK 0
#define ORA_EINVAL (-1)
#define ORA_ENOMEM (-2)
#define ORA_EINTERNAL (-3)
#define ORA_ECIGAR (-4)

#define ORA_OP_M 0
#define ORA_OP_I 1
#define ORA_OP_D 2

typedef struct {
    int32_t score1;
    int32_t score2;
    int32_t ref_begin1;
    int32_t ref_end1;
    int32_t read_begin1;
    int32_t read_end1;
    int32_t ref_end2;
    int32_t cigar_len;
    int32_t status;
} ora_result;

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

static int ora_check_scoring(const int8_t *W, int32_t A, int32_t O, int32_t X) {
    if (!W || A < 1 || A > 255) return ORA_EINVAL;
    if (X < 0 || O < X) return ORA_EINVAL;
    return ORA_OK;
}

/*
 * Local fill over all m x n cells, one column at a time (column j is H(.,j)).
 * colmax[j] = max_i H(i,j) (Algorithm (1), the "max" array; Fig. 1, bottom
 * row).  Returns score1 = max_j colmax[j] and the end cell by the first-column,
 * first-row rule; (-1,-1) when score1 = 0.
 */
int ora_fill(const uint8_t *q, int32_t m, const uint8_t *t, int32_t n,
             const int8_t *W, int32_t A, int32_t O, int32_t X,
             int32_t *colmax, int32_t *score1, int32_t *end_t, int32_t *end_q) {
    int rc = ora_check_scoring(W, A, O, X);
    if (rc) return rc;
    if (m < 0 || n < 0 || !colmax || !score1 || !end_t || !end_q) return ORA_EINVAL;
    *score1 = 0;
    *end_t = -1;
    *end_q = -1;
    if (m == 0 || n == 0) {
        for (int32_t j = 0; j < n; j++) colmax[j] = 0;
        return ORA_OK;
    }
    int32_t *Hcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)m); /* H(i, j-1) -> H(i, j) */
    int32_t *Ecol = (int32_t *)malloc(sizeof(int32_t) * (size_t)m); /* E(i, j-1) -> E(i, j) */
    if (!Hcol || !Ecol) {
        free(Hcol);
        free(Ecol);
        return ORA_ENOMEM;
    }
    for (int32_t i = 0; i < m; i++) {
        Hcol[i] = 0;       /* H(i, -1) = 0 */
        Ecol[i] = ORA_NEG; /* E(i, -1) = -inf */
    }
    int32_t best = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t h_diag = 0;  /* H(i-1, j-1); H(-1, .) = 0 */
        int32_t h_up = 0;    /* H(i-1, j) */
        int32_t f = ORA_NEG; /* F(-1, j) = -inf */
        int32_t cmax = 0;
        for (int32_t i = 0; i < m; i++) {
            if (q[i] >= A || t[j] >= A) {
                free(Hcol);
                free(Ecol);
                return ORA_EINVAL;
            }
            int32_t e = imax(Hcol[i] - O, Ecol[i] - X);
            f = imax(h_up - O, f - X);
            int32_t h = imax(0, h_diag + W[q[i] * A + t[j]]);
            h = imax(h, e);
            h = imax(h, f);
            h_diag = Hcol[i];
            Hcol[i] = h;
            Ecol[i] = e;
            h_up = h;
            cmax = imax(cmax, h);
        }
        colmax[j] = cmax;
        if (cmax > best) {
            /* the recorded column: the first row holding the new maximum */
            best = cmax;
            *end_t = j;
            for (int32_t i = 0; i < m; i++) {
                if (Hcol[i] == cmax) {
                    *end_q = i;
                    break;
                }
            }
        }
    }
    *score1 = best;
    free(Hcol);
    free(Ecol);
    return ORA_OK;
}

/*
 * Secondary score (Algorithm (2); Fig. 1 caption): mask the window
 * [end_t - L, end_t + L] of the max array and take the largest unmasked value
 * and its first column.  With no alignment (end_t < 0) nothing is masked.
 */
int ora_secondary(const int32_t *colmax, int32_t n, int32_t end_t, int32_t mask_len,
                  int32_t *score2, int32_t *ref_end2) {
    if (n < 0 || mask_len < 0 || !score2 || !ref_end2) return ORA_EINVAL;
    int32_t lo = 1, hi = 0; /* empty mask */
    if (end_t >= 0) {
        lo = end_t - mask_len;
        hi = end_t + mask_len;
    }
    int32_t s2 = 0, e2 = -1;
    for (int32_t j = 0; j < n; j++) {
        if (end_t >= 0 && j >= lo && j <= hi) continue;
        if (colmax[j] > s2) {
            s2 = colmax[j];
            e2 = j;
        }
    }
    *score2 = s2;
    *ref_end2 = e2;
    return ORA_OK;
}

/*
 * Begin by the reversed SW (Algorithm (1)): the same local fill on
 * reverse(q[0..end_q]) x reverse(t[0..end_t]); its maximum must equal score1,
 * and its end cell (first column, first row) maps back to the begin.
 */
int ora_begin(const uint8_t *q, const uint8_t *t, const int8_t *W, int32_t A,
              int32_t O, int32_t X, int32_t end_q, int32_t end_t, int32_t score1,
              int32_t *begin_q, int32_t *begin_t) {
    if (end_q < 0 || end_t < 0 || score1 <= 0) return ORA_EINVAL;
    int32_t mr = end_q + 1, nr = end_t + 1;
    uint8_t *qr = (uint8_t *)malloc((size_t)mr);
    uint8_t *tr = (uint8_t *)malloc((size_t)nr);
    int32_t *cm = (int32_t *)malloc(sizeof(int32_t) * (size_t)nr);
    if (!qr || !tr || !cm) {
        free(qr);
        free(tr);
        free(cm);
        return ORA_ENOMEM;
    }
    for (int32_t i = 0; i < mr; i++) qr[i] = q[end_q - i];
    for (int32_t j = 0; j < nr; j++) tr[j] = t[end_t - j];
    int32_t s, et, eq;
    int rc = ora_fill(qr, mr, tr, nr, W, A, O, X, cm, &s, &et, &eq);
    free(qr);
    free(tr);
    free(cm);
    if (rc) return rc;
    if (s != score1) return ORA_EINTERNAL;
    *begin_q = end_q - eq;
    *begin_t = end_t - et;
    return ORA_OK;
}

/* direction byte of one global-DP cell */
#define DIR_H_M 0
#define DIR_H_E 1
#define DIR_H_F 2
#define DIR_E_OPEN 4
#define DIR_F_OPEN 8

/*
 * Global Gotoh over the whole (la+1) x (lb+1) rectangle of qs x ts, then the
 * three-state traceback.  Cell (0,0) is the empty prefix; row 0 and column 0
 * follow the same recurrences with H(0,0) = 0 and -inf outside.  Writes the
 * run-length CIGAR (forward order) and the global score.
 */
int ora_cigar(const uint8_t *qs, int32_t la, const uint8_t *ts, int32_t lb,
              const int8_t *W, int32_t A, int32_t O, int32_t X,
              uint32_t *cigar, int32_t cigar_cap, int32_t *cigar_len, int32_t *score) {
    int rc = ora_check_scoring(W, A, O, X);
    if (rc) return rc;
    if (la < 1 || lb < 1 || !cigar_len || !score) return ORA_EINVAL;
    size_t rows = (size_t)la + 1, cols = (size_t)lb + 1;
    uint8_t *dir = (uint8_t *)malloc(rows * cols);
    int32_t *Hprev = (int32_t *)malloc(sizeof(int32_t) * cols);
    int32_t *Hcur = (int32_t *)malloc(sizeof(int32_t) * cols);
    int32_t *Fprev = (int32_t *)malloc(sizeof(int32_t) * cols);
    int32_t *Fcur = (int32_t *)malloc(sizeof(int32_t) * cols);
    uint8_t *ops = (uint8_t *)malloc(rows + cols);
    if (!dir || !Hprev || !Hcur || !Fprev || !Fcur || !ops) {
        free(dir); free(Hprev); free(Hcur); free(Fprev); free(Fcur); free(ops);
        return ORA_ENOMEM;
    }
    for (size_t i = 0; i < rows; i++) {
        int32_t e = ORA_NEG; /* E(i, 0) = -inf */
        for (size_t j = 0; j < cols; j++) {
            uint8_t d = 0;
            int32_t h, f;
            if (i == 0 && j == 0) {
                h = 0;
                f = ORA_NEG;
                e = ORA_NEG;
            } else {
                /* horizontal gap state (consumes target) */
                if (j > 0) {
                    int32_t open = Hcur[j - 1] - O, ext = e - X;
                    e = imax(open, ext);
                    if (e == open) d |= DIR_E_OPEN;
                } else {
                    e = ORA_NEG;
                }
                /* vertical gap state (consumes query) */
                if (i > 0) {
                    int32_t open = Hprev[j] - O, ext = Fprev[j] - X;
                    f = imax(open, ext);
                    if (f == open) d |= DIR_F_OPEN;
                } else {
                    f = ORA_NEG;
                }
                int32_t diag = ORA_NEG;
                if (i > 0 && j > 0) diag = Hprev[j - 1] + W[qs[i - 1] * A + ts[j - 1]];
                h = imax(diag, imax(e, f));
                if (i > 0 && j > 0 && h == diag) d |= DIR_H_M;
                else if (h == e) d |= DIR_H_E;
                else d |= DIR_H_F;
            }
            Hcur[j] = h;
            Fcur[j] = f;
            dir[i * cols + j] = d;
        }
        int32_t *tmp = Hprev; Hprev = Hcur; Hcur = tmp;
        tmp = Fprev; Fprev = Fcur; Fcur = tmp;
    }
    *score = Hprev[lb];
    /* traceback from (la, lb) in state H */
    size_t i = (size_t)la, j = (size_t)lb, nops = 0;
    int state = 0; /* 0 = H, 1 = E, 2 = F */
    while (i > 0 || j > 0) {
        uint8_t d = dir[i * cols + j];
        if (state == 0) {
            int src = d & 3;
            if (src == DIR_H_M) {
                ops[nops++] = ORA_OP_M;
                i--;
                j--;
            } else if (src == DIR_H_E) {
                state = 1;
            } else {
                state = 2;
            }
        } else if (state == 1) {
            ops[nops++] = ORA_OP_D;
            state = (d & DIR_E_OPEN) ? 0 : 1;
            j--;
        } else {
            ops[nops++] = ORA_OP_I;
            state = (d & DIR_F_OPEN) ? 0 : 2;
            i--;
        }
    }
    /* run-length encode in forward order */
    int32_t nrun = 0;
    size_t k = nops;
    while (k > 0) {
        uint8_t op = ops[k - 1];
        uint32_t len = 0;
        while (k > 0 && ops[k - 1] == op) {
            len++;
            k--;
        }
        if (cigar && nrun < cigar_cap) cigar[nrun] = (len << 4) | op;
        nrun++;
    }
    *cigar_len = nrun;
    free(dir); free(Hprev); free(Hcur); free(Fprev); free(Fcur); free(ops);
    if (cigar_cap >= 0 && nrun > cigar_cap) return ORA_ECIGAR;
    return ORA_OK;
}

/* the four steps for one pair (Results, Usage: the optimum's score, position
 * and alignment; the second-best score and its end column) */
int ora_align(const uint8_t *q, int32_t m, const uint8_t *t, int32_t n,
              const int8_t *W, int32_t A, int32_t O, int32_t X, int32_t mask_len,
              int32_t *colmax_out, uint32_t *cigar, int32_t cigar_cap, ora_result *res) {
    if (!res) return ORA_EINVAL;
    memset(res, 0, sizeof(*res));
    res->ref_begin1 = res->ref_end1 = res->read_begin1 = res->read_end1 = res->ref_end2 = -1;
    int rc = ora_check_scoring(W, A, O, X);
    if (rc || m < 0 || n < 0) return res->status = (rc ? rc : ORA_EINVAL);
    int32_t *cm = colmax_out;
    if (!cm) {
        cm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!cm) return res->status = ORA_ENOMEM;
    }
    int32_t s1, et, eq;
    rc = ora_fill(q, m, t, n, W, A, O, X, cm, &s1, &et, &eq);
    if (rc) goto done;
    res->score1 = s1;
    res->ref_end1 = et;
    res->read_end1 = eq;
    int32_t L = mask_len >= 0 ? mask_len : imax(m / 2, 15);
    rc = ora_secondary(cm, n, et, L, &res->score2, &res->ref_end2);
    if (rc || s1 <= 0) goto done;
    int32_t bq, bt;
    rc = ora_begin(q, t, W, A, O, X, eq, et, s1, &bq, &bt);
    if (rc) goto done;
    res->read_begin1 = bq;
    res->ref_begin1 = bt;
    int32_t glob;
    rc = ora_cigar(q + bq, eq - bq + 1, t + bt, et - bt + 1, W, A, O, X, cigar, cigar_cap,
                   &res->cigar_len, &glob);
    if (rc == ORA_OK && glob != s1) rc = ORA_EINTERNAL;
done:
    if (cm != colmax_out) free(cm);
    res->status = rc;
    return rc;
}

/* ---- batch over pairs, one pthread per core ------------------------------ */

typedef struct {
    int32_t npairs;
    const uint8_t *qa;
    const int64_t *qoff;
    const int32_t *qlen;
    const uint8_t *ta;
    const int64_t *toff;
    const int32_t *tlen;
    const int8_t *W;
    int32_t A, O, X, mask_len;
    ora_result *res;
    uint32_t *cigar;
    int32_t cigar_stride;
    int32_t *colmax;
    const int64_t *colmax_off;
    volatile int32_t next;
    pthread_mutex_t lock;
} ora_batch;

static void *ora_worker(void *arg) {
    ora_batch *b = (ora_batch *)arg;
    for (;;) {
        pthread_mutex_lock(&b->lock);
        int32_t p = b->next++;
        pthread_mutex_unlock(&b->lock);
        if (p >= b->npairs) break;
        int32_t *cm = b->colmax ? b->colmax + b->colmax_off[p] : NULL;
        uint32_t *cg = b->cigar ? b->cigar + (size_t)p * (size_t)b->cigar_stride : NULL;
        ora_align(b->qa + b->qoff[p], b->qlen[p], b->ta + b->toff[p], b->tlen[p], b->W, b->A,
                  b->O, b->X, b->mask_len, cm, cg, b->cigar ? b->cigar_stride : -1, &b->res[p]);
    }
    return NULL;
}

/* Aligns every pair; returns 0, or the first non-zero pair status. */
int ora_align_batch(int32_t npairs, const uint8_t *qa, const int64_t *qoff, const int32_t *qlen,
                    const uint8_t *ta, const int64_t *toff, const int32_t *tlen,
                    const int8_t *W, int32_t A, int32_t O, int32_t X, int32_t mask_len,
                    ora_result *res, uint32_t *cigar, int32_t cigar_stride,
                    int32_t *colmax, const int64_t *colmax_off, int32_t nthreads) {
    if (npairs < 0 || !res || nthreads < 1) return ORA_EINVAL;
    ora_batch b;
    b.npairs = npairs; b.qa = qa; b.qoff = qoff; b.qlen = qlen;
    b.ta = ta; b.toff = toff; b.tlen = tlen; b.W = W; b.A = A; b.O = O; b.X = X;
    b.mask_len = mask_len; b.res = res; b.cigar = cigar; b.cigar_stride = cigar_stride;
    b.colmax = colmax; b.colmax_off = colmax_off; b.next = 0;
    pthread_mutex_init(&b.lock, NULL);
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int32_t started = 0;
    for (int32_t k = 1; k < nthreads; k++) {
        if (pthread_create(&th[started], NULL, ora_worker, &b) == 0) started++;
    }
    ora_worker(&b);
    for (int32_t k = 0; k < started; k++) pthread_join(th[k], NULL);
    pthread_mutex_destroy(&b.lock);
    for (int32_t p = 0; p < npairs; p++)
        if (res[p].status) return res[p].status;
    return ORA_OK;
}
