"""Brute-force enumeration of alignments, used to pin the oracle.

Nothing here runs a dynamic program.  Local alignments are enumerated as
explicit transcripts (sequences of M / I / D operations) and scored by the
textbook affine rule: the sum of substitution scores over M columns minus,
for every maximal run of I or of D of length k, open + (k-1) * extend.  The
per-cell, per-column and optimal quantities the method defines are then read
off the enumerated set.  Only usable for sequences of length <= 7.
"""
from __future__ import annotations

M, I, D = 0, 1, 2


def transcript_score(ops, qs, ts, W, gap_open, gap_extend):
    """Score of an op string over q-substring qs and t-substring ts."""
    s = 0
    i = j = 0
    prev = None
    for op in ops:
        if op == M:
            s += int(W[qs[i]][ts[j]])
            i += 1
            j += 1
        elif op == I:
            s -= gap_extend if prev == I else gap_open
            i += 1
        else:
            s -= gap_extend if prev == D else gap_open
            j += 1
        prev = op
    assert i == len(qs) and j == len(ts)
    return s


def enumerate_local(q, t, W, gap_open, gap_extend):
    """Every transcript that starts with an M column, with its score, start cell
    (a, c) and end cell (i, j) = (last query index used, last target index used).

    Yields (score, a, c, i, j).  Transcripts may end in a gap run (a trailing gap
    leaves the last used indices where the DP cell (i, j) keeps them).
    """
    m, n = len(q), len(t)
    out = []
    for a in range(m):
        for c in range(n):
            # DFS over (i, j, prev_op, score) after the first M at (a, c)
            stack = [(a, c, M, int(W[q[a]][t[c]]))]
            while stack:
                i, j, prev, s = stack.pop()
                out.append((s, a, c, i, j))
                if i + 1 < m and j + 1 < n:
                    stack.append((i + 1, j + 1, M, s + int(W[q[i + 1]][t[j + 1]])))
                if i + 1 < m:
                    stack.append((i + 1, j, I, s - (gap_extend if prev == I else gap_open)))
                if j + 1 < n:
                    stack.append((i, j + 1, D, s - (gap_extend if prev == D else gap_open)))
    return out


def local_summary(q, t, W, gap_open, gap_extend):
    """Quantities the method defines, read off the enumeration.

    H[i][j]  = max(0, best transcript ending at (i, j))
    colmax[j] = max_i H[i][j]
    score1 = max over everything (0 for the empty alignment)
    end    = lexicographically smallest (j, i) among transcripts scoring score1
    begin  = largest (c, a) among transcripts scoring score1 that end at `end`
    """
    m, n = len(q), len(t)
    H = [[0] * n for _ in range(m)]
    al = enumerate_local(q, t, W, gap_open, gap_extend)
    for s, a, c, i, j in al:
        if s > H[i][j]:
            H[i][j] = s
    colmax = [max((H[i][j] for i in range(m)), default=0) for j in range(n)]
    score1 = max(colmax, default=0)
    if score1 <= 0:
        return dict(H=H, colmax=colmax, score1=0, end=(-1, -1), begin=(-1, -1))
    best = [(j, i) for s, a, c, i, j in al if s == score1]
    ej, ei = min(best)
    starts = [(c, a) for s, a, c, i, j in al if s == score1 and (i, j) == (ei, ej)]
    bc, ba = max(starts)
    return dict(H=H, colmax=colmax, score1=score1, end=(ei, ej), begin=(ba, bc))


def enumerate_global(qs, ts):
    """All op strings aligning qs and ts end to end."""
    la, lb = len(qs), len(ts)
    out = []

    def rec(i, j, ops):
        if i == la and j == lb:
            out.append(tuple(ops))
            return
        if i < la and j < lb:
            ops.append(M)
            rec(i + 1, j + 1, ops)
            ops.pop()
        if i < la:
            ops.append(I)
            rec(i + 1, j, ops)
            ops.pop()
        if j < lb:
            ops.append(D)
            rec(i, j + 1, ops)
            ops.pop()

    rec(0, 0, [])
    return out


def canonical_global(qs, ts, W, gap_open, gap_extend):
    """Optimal global score and the canonical optimal transcript.

    The canonical one is chosen walking backwards from the end: after an M (or
    at the end) prefer M, then D, then I; after a D prefer M, then I, then D
    (a gap run is closed as early as possible, then the H-state order applies,
    where a second D cannot follow an opened gap when open > extend); after an
    I prefer M, then D, then I.  Each choice keeps only the optimal transcripts
    consistent with the ops chosen so far.  Valid for open > extend.
    """
    alls = enumerate_global(qs, ts)
    scored = [(transcript_score(o, qs, ts, W, gap_open, gap_extend), o) for o in alls]
    best = max(s for s, _ in scored)
    cands = [o for s, o in scored if s == best]
    suffix = []  # chosen ops, backwards
    prev = None
    while True:
        k = len(suffix)
        live = [o for o in cands if len(o) >= k and (k == 0 or tuple(o[len(o) - k:]) == tuple(reversed(suffix)))]
        if any(len(o) == k for o in live):
            break
        order = [M, I, D] if prev == D else [M, D, I]
        for op in order:
            if any(o[len(o) - k - 1] == op for o in live if len(o) > k):
                suffix.append(op)
                prev = op
                break
        cands = live
    return best, list(reversed(suffix))


def runs(ops):
    """Run-length encode an op list into [(len, op)]."""
    out = []
    for op in ops:
        if out and out[-1][1] == op:
            out[-1] = (out[-1][0] + 1, op)
        else:
            out.append((1, op))
    return out
