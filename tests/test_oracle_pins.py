"""Pins of the CPU oracle against things other than itself.

Brute-force enumeration of transcripts (tests/brute_force.py), closed forms,
textbook special cases (Kadane's maximum subarray for ungapped local alignment,
Levenshtein distance for unit-cost global alignment), a worked textbook example
(tests/golden/), and invariants.  None of these calls the oracle's own
recurrence a second time.
"""
import json
import os

import numpy as np
import pytest

import oracle
from brute_force import canonical_global, local_summary, runs, transcript_score

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dna_matrix(match, mismatch, A=4):
    W = np.full((A, A), mismatch, dtype=np.int8)
    np.fill_diagonal(W, match)
    return W


def random_case(rng, max_len=6):
    A = int(rng.integers(2, 5))
    m = int(rng.integers(1, max_len + 1))
    n = int(rng.integers(1, max_len + 1))
    q = rng.integers(0, A, m).astype(np.uint8)
    t = rng.integers(0, A, n).astype(np.uint8)
    if rng.random() < 0.5:
        W = dna_matrix(int(rng.integers(1, 5)), -int(rng.integers(1, 5)), A)
    else:
        W = rng.integers(-4, 5, (A, A)).astype(np.int8)  # possibly asymmetric
        W[0, 0] = max(W[0, 0], 1)
    X = int(rng.integers(1, 4))
    O = X + int(rng.integers(0, 4))
    return q, t, W, O, X


def test_fill_and_begin_match_brute_force():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(300):
        q, t, W, O, X = random_case(rng)
        bf = local_summary(list(q), list(t), W, O, X)
        cm, s1, et, eq = oracle.fill(q, t, W, O, X)
        assert s1 == bf["score1"]
        assert list(cm) == bf["colmax"]
        assert (eq, et) == bf["end"]
        if s1 > 0:
            bq, bt = oracle.begin(q, t, W, O, X, eq, et, s1)
            assert (bq, bt) == bf["begin"]
            checked += 1
    assert checked > 100


def test_brute_force_length_seven():
    rng = np.random.default_rng(7)
    for _ in range(4):
        q = rng.integers(0, 3, 7).astype(np.uint8)
        t = rng.integers(0, 3, 7).astype(np.uint8)
        W = dna_matrix(2, -1, 3)
        bf = local_summary(list(q), list(t), W, 2, 1)
        r = oracle.align(q, t, W, 2, 1)
        assert r["score1"] == bf["score1"]
        assert list(r["colmax"]) == bf["colmax"]
        if r["score1"] > 0:
            assert (r["read_end1"], r["ref_end1"]) == bf["end"]
            assert (r["read_begin1"], r["ref_begin1"]) == bf["begin"]


def rescore(r, q, t, W, O, X):
    ops = [op for n_, op in r["cigar"] for _ in range(n_)]
    qs = list(q[r["read_begin1"]:r["read_end1"] + 1])
    ts = list(t[r["ref_begin1"]:r["ref_end1"] + 1])
    return transcript_score(ops, qs, ts, W, O, X), ops


def test_cigar_is_optimal_and_canonical():
    rng = np.random.default_rng(3)
    n_canon = 0
    for _ in range(250):
        q, t, W, O, X = random_case(rng)
        r = oracle.align(q, t, W, O, X)
        if r["score1"] == 0:
            assert r["cigar"] == [] and r["ref_begin1"] == -1 and r["read_end1"] == -1
            continue
        s, ops = rescore(r, q, t, W, O, X)
        assert s == r["score1"]
        assert sum(1 for o in ops if o != 2) == r["read_end1"] - r["read_begin1"] + 1
        assert sum(1 for o in ops if o != 1) == r["ref_end1"] - r["ref_begin1"] + 1
        qs = list(q[r["read_begin1"]:r["read_end1"] + 1])
        ts = list(t[r["ref_begin1"]:r["ref_end1"] + 1])
        if O > X and len(qs) + len(ts) <= 11:
            best, canon = canonical_global(qs, ts, W, O, X)
            assert best == r["score1"]
            assert runs(canon) == r["cigar"]
            n_canon += 1
    assert n_canon > 50


def test_cigar_canonical_choice_on_gapped_pairs():
    # pairs built to need a gap, so that the gap placement rule is exercised
    rng = np.random.default_rng(11)
    W = dna_matrix(2, -3)
    n_gap = 0
    for _ in range(120):
        la = int(rng.integers(3, 6))
        qs = rng.integers(0, 4, la).astype(np.uint8)
        ins = rng.integers(0, 4, int(rng.integers(1, 3))).astype(np.uint8)
        cut = int(rng.integers(1, la))
        ts = np.concatenate([qs[:cut], ins, qs[cut:]])
        if rng.random() < 0.5:
            qs, ts = ts, qs
        for O, X in ((3, 1), (4, 2), (2, 1)):
            best, canon = canonical_global(list(qs), list(ts), W, O, X)
            got, sc = oracle.cigar(qs, ts, W, O, X)
            assert sc == best
            assert got == runs(canon)
            n_gap += any(op != 0 for op in canon)
    assert n_gap > 100


def test_textbook_worked_example():
    with open(os.path.join(GOLDEN, "sw_textbook_example.json")) as f:
        g = json.load(f)
    code = {c: k for k, c in enumerate(g["alphabet"])}
    q = np.array([code[c] for c in g["query"]], dtype=np.uint8)
    t = np.array([code[c] for c in g["target"]], dtype=np.uint8)
    W = dna_matrix(g["match"], g["mismatch"])
    r = oracle.align(q, t, W, g["gap_open"], g["gap_extend"])
    e = g["expected"]
    for k in ("score1", "read_begin1", "read_end1", "ref_begin1", "ref_end1"):
        assert r[k] == e[k], k
    assert oracle.cigar_string(r["cigar"]) == e["cigar"]


def test_self_alignment_closed_form():
    rng = np.random.default_rng(5)
    for m in (1, 2, 5, 17, 64, 150):
        q = rng.integers(0, 4, m).astype(np.uint8)
        W = dna_matrix(2, -2)
        r = oracle.align(q, q, W, 3, 1)
        assert r["score1"] == 2 * m
        assert (r["read_begin1"], r["read_end1"], r["ref_begin1"], r["ref_end1"]) == (0, m - 1, 0, m - 1)
        assert r["cigar"] == [(m, 0)]


def test_self_alignment_general_matrix():
    # self score is the sum of diagonal entries when every diagonal entry is the
    # row maximum and strictly positive
    rng = np.random.default_rng(6)
    A = 20
    W = rng.integers(-4, 4, (A, A)).astype(np.int8)
    W = np.minimum(W, W.T)
    np.fill_diagonal(W, rng.integers(5, 12, A))
    q = rng.integers(0, A, 40).astype(np.uint8)
    r = oracle.align(q, q, W, 11, 1)
    assert r["score1"] == int(sum(int(W[a, a]) for a in q))


def test_disjoint_alphabets_score_zero():
    W = dna_matrix(2, -2)
    q = np.array([0, 1, 0, 1, 1, 0], dtype=np.uint8)
    t = np.array([2, 3, 3, 2, 2, 3, 2], dtype=np.uint8)
    r = oracle.align(q, t, W, 3, 1)
    assert r["score1"] == 0 and r["score2"] == 0
    assert (r["ref_end1"], r["read_end1"], r["ref_begin1"], r["read_begin1"], r["ref_end2"]) == (-1,) * 5
    assert r["cigar"] == []
    assert not r["colmax"].any()


def test_single_shared_letter():
    W = dna_matrix(2, -2)
    q = np.array([0, 0, 1, 0, 0], dtype=np.uint8)      # one C among A
    t = np.array([2, 3, 1, 2, 3, 2], dtype=np.uint8)   # one C among G/T
    r = oracle.align(q, t, W, 3, 1)
    assert r["score1"] == 2
    assert (r["read_end1"], r["ref_end1"], r["read_begin1"], r["ref_begin1"]) == (2, 2, 2, 2)


@pytest.mark.parametrize("O,X", [(3, 1), (4, 2), (11, 1), (5, 5)])
def test_forced_gap_closed_form(O, X):
    # q = Xs Ys over {A,C}; t = Xs Z Ys with Z of G only: any alignment that uses
    # both halves must gap all of Z (one run), so
    # score1 = max(2(|Xs|+|Ys|) - (O + (g-1) X), 2|Xs|, 2|Ys|).
    rng = np.random.default_rng(O * 10 + X)
    W = dna_matrix(2, -2)
    for _ in range(30):
        a, b, g = (int(v) for v in rng.integers(4, 30, 3))
        xs = rng.integers(0, 2, a).astype(np.uint8)
        ys = rng.integers(0, 2, b).astype(np.uint8)
        z = np.full(g, 2, dtype=np.uint8)
        q = np.concatenate([xs, ys])
        t = np.concatenate([xs, z, ys])
        want = max(2 * (a + b) - (O + (g - 1) * X), 2 * a, 2 * b)
        assert oracle.align(q, t, W, O, X)["score1"] == want


def kadane_ungapped(q, t, W):
    """Best ungapped local alignment: maximum subarray along every diagonal."""
    best = 0
    m, n = len(q), len(t)
    for d in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + d
            if 0 <= j < n:
                run = max(0, run + int(W[q[i], t[j]]))
                best = max(best, run)
    return best


def test_ungapped_special_case_is_kadane():
    rng = np.random.default_rng(9)
    for _ in range(40):
        A = int(rng.integers(2, 6))
        W = rng.integers(-5, 5, (A, A)).astype(np.int8)
        q = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        t = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        big = 127  # a gap can never pay back: |q| * max W < open
        if len(q) * max(int(W.max()), 0) >= big:
            continue
        _, s1, _, _ = oracle.fill(q, t, W, big, 1)
        assert s1 == kadane_ungapped(q, t, W)


def levenshtein(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def test_global_unit_cost_is_levenshtein():
    rng = np.random.default_rng(13)
    W = dna_matrix(0, -1)
    for _ in range(60):
        a = rng.integers(0, 4, int(rng.integers(1, 25))).astype(np.uint8)
        b = rng.integers(0, 4, int(rng.integers(1, 25))).astype(np.uint8)
        runs_, sc = oracle.cigar(a, b, W, 1, 1)
        assert sc == -levenshtein(list(a), list(b))
        assert sum(n for n, op in runs_ if op != 2) == len(a)
        assert sum(n for n, op in runs_ if op != 1) == len(b)


def test_swap_invariance_with_transposed_matrix():
    rng = np.random.default_rng(17)
    for _ in range(60):
        A = int(rng.integers(2, 6))
        W = rng.integers(-4, 5, (A, A)).astype(np.int8)
        q = rng.integers(0, A, int(rng.integers(1, 50))).astype(np.uint8)
        t = rng.integers(0, A, int(rng.integers(1, 50))).astype(np.uint8)
        X = int(rng.integers(0, 3))
        O = X + int(rng.integers(0, 4))
        a = oracle.fill(q, t, W, O, X)[1]
        b = oracle.fill(t, q, W.T.copy(), O, X)[1]
        assert a == b >= 0


def test_end_tie_rule_on_repeated_query():
    # the query occurs twice exactly: the end is the first copy's last column
    rng = np.random.default_rng(21)
    W = dna_matrix(2, -2)
    q = rng.integers(0, 4, 30).astype(np.uint8)
    t = np.concatenate([rng.integers(0, 4, 40), q, rng.integers(0, 4, 50), q,
                        rng.integers(0, 4, 10)]).astype(np.uint8)
    r = oracle.align(q, t, W, 3, 1)
    assert r["score1"] == 60
    assert r["ref_end1"] == 40 + 29 and r["read_end1"] == 29
    assert r["ref_begin1"] == 40 and r["read_begin1"] == 0
    # second copy is outside the default mask (max(30/2, 15) = 15): score2 = 60
    assert r["score2"] == 60 and r["ref_end2"] == 40 + 30 + 50 + 29
    # a mask wider than the distance between copies hides the second one
    r2 = oracle.align(q, t, W, 3, 1, mask_len=90)
    assert r2["score2"] < 60


def test_invariants_on_random_pairs():
    rng = np.random.default_rng(23)
    W = dna_matrix(2, -2)
    for _ in range(50):
        m = int(rng.integers(1, 80))
        n = int(rng.integers(1, 200))
        q = rng.integers(0, 4, m).astype(np.uint8)
        t = rng.integers(0, 4, n).astype(np.uint8)
        t[: min(m, n)] = q[: min(m, n)] if rng.random() < 0.5 else t[: min(m, n)]
        r = oracle.align(q, t, W, 3, 1)
        cm = r["colmax"]
        assert r["score1"] >= 0 and (cm >= 0).all()
        assert cm.max(initial=0) == r["score1"]
        if r["score1"] > 0:
            assert cm[r["ref_end1"]] == r["score1"]
            assert (cm[: r["ref_end1"]] < r["score1"]).all()
            assert r["read_begin1"] <= r["read_end1"] and r["ref_begin1"] <= r["ref_end1"]
            s, _ = rescore(r, q, t, W, 3, 1)
            assert s == r["score1"]
        assert r["score2"] <= r["score1"]


def test_batch_matches_single_calls():
    rng = np.random.default_rng(29)
    W = dna_matrix(2, -2)
    qs = [rng.integers(0, 4, int(rng.integers(0, 60))).astype(np.uint8) for _ in range(40)]
    ts = [rng.integers(0, 4, int(rng.integers(0, 120))).astype(np.uint8) for _ in range(40)]
    qa, ta = np.concatenate(qs), np.concatenate(ts)
    qlen = np.array([len(x) for x in qs]); tlen = np.array([len(x) for x in ts])
    qoff = np.concatenate([[0], np.cumsum(qlen)[:-1]]); toff = np.concatenate([[0], np.cumsum(tlen)[:-1]])
    res, cg, (cm, cmoff) = oracle.align_batch(qa, qoff, qlen, ta, toff, tlen, W, 3, 1,
                                             nthreads=3, cigar_stride=200, colmax=True)
    for p in range(40):
        r = oracle.align(qs[p], ts[p], W, 3, 1)
        for k in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1",
                  "ref_end2", "cigar_len"):
            assert res[k][p] == r[k]
        assert oracle.decode_cigar(cg[p, : r["cigar_len"]]) == r["cigar"]
        assert (cm[cmoff[p]: cmoff[p] + tlen[p]] == r["colmax"]).all()


def _all_strings(A, max_len):
    out = [[]]
    for L in range(1, max_len + 1):
        for k in range(A ** L):
            s, v = [], k
            for _ in range(L):
                s.append(v % A)
                v //= A
            out.append(s)
    return out[1:]


@pytest.mark.parametrize("match,mismatch,O,X", [(2, -3, 3, 1), (2, -1, 2, 1), (1, -1, 3, 1),
                                                (3, -2, 4, 2)])
def test_cigar_canonical_exhaustive_small(match, mismatch, O, X):
    # every pair of strings of length <= 3 over three letters: all tie patterns
    # between M, D and I, and between opening and extending a gap, occur here
    W = dna_matrix(match, mismatch, 3)
    strs = _all_strings(3, 3)
    for qs in strs:
        for ts in strs:
            best, canon = canonical_global(qs, ts, W, O, X)
            got, sc = oracle.cigar(np.array(qs, np.uint8), np.array(ts, np.uint8), W, O, X)
            assert sc == best
            assert got == runs(canon), (qs, ts)


def test_d_preferred_over_i_on_tie():
    # AC against CA: I M D and D M I both score -4; walking back from the end,
    # the horizontal gap state (D) is preferred, giving 1I1M1D
    W = dna_matrix(2, -3, 2)
    got, sc = oracle.cigar(np.array([0, 1], np.uint8), np.array([1, 0], np.uint8), W, 3, 1)
    assert sc == -4 and oracle.cigar_string(got) == "1I1M1D"


def _two_copies(m1, m2, gap, rng):
    """target = pad + Q[:m1] + spacer + Q[:m2] + pad over {A,C} vs query Q over {A,C}.

    The spacer and pads are G/T only, so each copy scores 2 * its length.
    """
    m = max(m1, m2)
    q = rng.integers(0, 2, m).astype(np.uint8)
    pad = lambda k: rng.integers(2, 4, k).astype(np.uint8)
    t = np.concatenate([pad(20), q[:m1], pad(gap), q[:m2], pad(20)])
    return q, t, 20 + m1 - 1, 20 + m1 + gap + m2 - 1


def test_secondary_mask_bounds_right_side():
    rng = np.random.default_rng(31)
    W = dna_matrix(2, -2)
    q, t, e1, e2 = _two_copies(40, 40, 30, rng)
    d = e2 - e1
    r = oracle.align(q, t, W, 3, 1, mask_len=d)       # e2 = e1 + L: masked
    assert r["ref_end1"] == e1 and r["score1"] == 80 and r["score2"] < 80
    r = oracle.align(q, t, W, 3, 1, mask_len=d - 1)   # e2 = e1 + L + 1: visible
    assert r["score2"] == 80 and r["ref_end2"] == e2


def test_secondary_mask_bounds_left_side():
    rng = np.random.default_rng(37)
    W = dna_matrix(2, -2)
    q, t, e1, e2 = _two_copies(25, 40, 30, rng)       # the right copy is primary
    d = e2 - e1
    r = oracle.align(q, t, W, 3, 1, mask_len=d)       # e1 = e2 - L: masked
    assert r["ref_end1"] == e2 and r["score1"] == 80 and r["score2"] < 50
    r = oracle.align(q, t, W, 3, 1, mask_len=d - 1)   # e1 = e2 - L - 1: visible
    assert r["score2"] == 50 and r["ref_end2"] == e1


def test_secondary_tie_takes_first_column():
    rng = np.random.default_rng(41)
    W = dna_matrix(2, -2)
    m = 30
    q = rng.integers(0, 2, m).astype(np.uint8)
    pad = lambda k: rng.integers(2, 4, k).astype(np.uint8)
    # primary: a full copy; two equal partial copies (20 letters) further right.
    # The primary's trailing-gap tail in the max array (60 - 3 - (k - 1) at k
    # columns past its end) must lie inside the mask, hence mask_len = 60 and
    # the copies start 70 columns after the primary.
    t = np.concatenate([pad(10), q, pad(70), q[:20], pad(40), q[:20], pad(10)])
    r = oracle.align(q, t, W, 3, 1, mask_len=60)
    assert r["score1"] == 60 and r["score2"] == 40
    assert r["ref_end2"] == 10 + m + 70 + 20 - 1
