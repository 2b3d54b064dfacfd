"""CPU checks of the library's host-side geometry rules, compiled from the
library's own header with g++ (tests/host_rules_shim.cpp):

* the reversed fill's window and its band [-Gn, G] (gap letters bounded by the
  score; the reversed pass for the begin, "Algorithm and implementation") hold
  every optimal path the oracle reports, and are exact on closed-form gapped
  pairs;
* the traceback band [dlo, dhi] (the banded global alignment between begin and
  end, same section) holds the oracle's CIGAR path, and is exact on the same
  pairs;
* the traceback class routing: widths map to the anti-diagonal classes, bands
  wider than 512 diagonals go to the 16-bit rectangle whenever its values and
  scratch fit (never to the ring kernel then), and the rectangle is never
  chosen for values or regions it cannot hold.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

T16_FIRST, RING = 5, 4


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("cuda_runtime.h not found")
    return inc


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_rules") / "libhostrules.so")
    subprocess.run([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-w",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1208_6350_gb300", "csrc"),
                    "-I", _cuda_include(),
                    os.path.join(HERE, "host_rules_shim.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    i32 = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    for name, args in (("hr_reverse_window", [i32, P, i32, i32, i32, i32, i32]),
                       ("hr_reverse_gap_bound", [i32, P, i32, i32, i32, i32]),
                       ("hr_reverse_gap_bound_rows", [i32, P, i32, i32, i32, i32]),
                       ("hr_band_range", [i32, P, i32, i32, i32, i32, i32, ip, ip]),
                       ("hr_trace_class", [i32, P, i32, i32, i32, i32, i32, i32, ip, ip])):
        getattr(L, name).argtypes = args
        getattr(L, name).restype = i32
    L.hr_t16_need_words.argtypes = [i32, i32, i32]
    L.hr_t16_need_words.restype = ctypes.c_longlong
    L.hr_pick_class.argtypes = [i32, P, i32, i32, P, i32, i32, i32]
    L.hr_pick_class.restype = i32
    L.hr_fill_class_mask.argtypes = [i32, P, i32, i32, P, i32, i32, i32, i32]
    L.hr_fill_class_mask.restype = ctypes.c_uint
    L.hr_batch_status.argtypes = [i32, ctypes.c_ulonglong, i32, ctypes.c_ulonglong, ctypes.c_longlong]
    L.hr_batch_status.restype = i32
    return L


class Rules:
    """The rules for one scoring scheme (W is A x A int8, row = query letter)."""

    def __init__(self, L, W, O, X):
        self.L, self.O, self.X = L, O, X
        self.W = np.ascontiguousarray(W, dtype=np.int8)
        self.A = self.W.shape[0]
        self.p = self.W.ctypes.data_as(ctypes.c_void_p)

    def window(self, eq, et, s1):
        return self.L.hr_reverse_window(self.A, self.p, self.O, self.X, eq, et, s1)

    def G(self, eq, s1):
        return self.L.hr_reverse_gap_bound(self.A, self.p, self.O, self.X, eq, s1)

    def Gn(self, eq, s1):
        return self.L.hr_reverse_gap_bound_rows(self.A, self.p, self.O, self.X, eq, s1)

    def band(self, la, lb, s1):
        lo, hi = ctypes.c_int(), ctypes.c_int()
        self.L.hr_band_range(self.A, self.p, self.O, self.X, la, lb, s1, ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value

    def trace_class(self, la, lb, s1, small=False):
        lo, hi = ctypes.c_int(), ctypes.c_int()
        c = self.L.hr_trace_class(self.A, self.p, self.O, self.X, la, lb, s1, int(small),
                                  ctypes.byref(lo), ctypes.byref(hi))
        return c, hi.value - lo.value + 1


def dna(match, mismatch, A=4):
    W = np.full((A, A), mismatch, dtype=np.int8)
    np.fill_diagonal(W, match)
    return W


def protein_like(rng, A=20):
    W = rng.integers(-4, 4, (A, A))
    W = np.triu(W) + np.triu(W, 1).T
    np.fill_diagonal(W, rng.integers(4, 12, A))
    return W.astype(np.int8)


def mutate(rng, s, A, sub, indel, max_run=6):
    out = []
    i = 0
    while i < len(s):
        r = rng.random()
        if r < indel / 2:
            out.extend(rng.integers(0, A, int(rng.integers(1, max_run + 1))).tolist())
        elif r < indel:
            i += int(rng.integers(1, max_run + 1))
            continue
        out.append(int(rng.integers(0, A)) if rng.random() < sub else int(s[i]))
        i += 1
    return np.array(out if out else [0], dtype=np.uint8)


def path_diagonals(cigar):
    """Diagonals (target minus query letters consumed) of every cell of a CIGAR
    path, forward from the begin and backward from the end."""
    fwd, bwd = [0], [0]
    i = j = 0
    for n, op in cigar:
        for _ in range(n):
            i += op != 2   # M and I consume a query letter
            j += op != 1   # M and D consume a target letter
            fwd.append(j - i)
    i = j = 0
    for n, op in reversed(cigar):
        for _ in range(n):
            i += op != 2
            j += op != 1
            bwd.append(j - i)
    return fwd, bwd


def check_pair(R, q, t):
    r = oracle.align(q, t, R.W, R.O, R.X)
    s1 = r["score1"]
    if s1 <= 0:
        return False
    eq, et, bq, bt = r["read_end1"], r["ref_end1"], r["read_begin1"], r["ref_begin1"]
    cig = r["cigar"]
    la, lb = eq - bq + 1, et - bt + 1
    # the reversed fill scans columns [end_t + 1 - window, end_t]
    assert bt >= et + 1 - R.window(eq, et, s1)
    # its band [-Gn, G] below/above the reversed main diagonal
    G, Gn = R.G(eq, s1), R.Gn(eq, s1)
    gaps_t = sum(n for n, op in cig if op == 2)
    gaps_q = sum(n for n, op in cig if op == 1)
    assert gaps_t + gaps_q <= G and gaps_q <= Gn
    fwd, bwd = path_diagonals(cig)
    assert min(bwd) >= -Gn and max(bwd) <= G
    # the traceback band between begin and end
    dlo, dhi = R.band(la, lb, s1)
    assert dlo <= min(fwd) and max(fwd) <= dhi
    assert fwd[-1] == lb - la
    return True


@pytest.mark.parametrize("kind", ["dna", "protein"])
def test_bounds_hold_the_oracle_paths_on_related_pairs(lib, kind):
    rng = np.random.default_rng(11 if kind == "dna" else 12)
    checked = 0
    for it in range(120):
        if kind == "dna":
            A = 4
            W = dna(int(rng.integers(1, 4)), -int(rng.integers(1, 5)))
        else:
            A = 20
            W = protein_like(rng)
        X = int(rng.integers(1, 4))
        O = X + int(rng.integers(0, 10))
        R = Rules(lib, W, O, X)
        n = int(rng.integers(5, 300))
        base = rng.integers(0, A, n).astype(np.uint8)
        q = mutate(rng, base, A, sub=rng.random() * 0.2, indel=rng.random() * 0.15)
        t = np.concatenate([rng.integers(0, A, int(rng.integers(0, 40))).astype(np.uint8),
                            mutate(rng, base, A, sub=0.05, indel=0.05),
                            rng.integers(0, A, int(rng.integers(0, 40))).astype(np.uint8)])
        checked += check_pair(R, q, t)
    assert checked > 100


@pytest.mark.parametrize("g", [1, 2, 5, 8])
def test_bounds_are_exact_on_one_gap_pairs(lib, g):
    """Query x+y against target x+z+y (z: g letters that match nothing): the
    optimum is the one-gap path, score (a+b)m - O - (g-1)X; the forward bound
    on gap letters, the reversed band's upper edge and the traceback band
    are then exactly g (the gap count follows from the score).
    Swapping the roles gives the rows bound Gn = g."""
    rng = np.random.default_rng(100 + g)
    A, m, O, X = 5, 2, 5, 2
    W = dna(m, -3, A)
    W[4, 4] = -3  # letter 4 matches nothing
    R = Rules(lib, W, O, X)
    a, b = 40, 50
    x = rng.integers(0, 4, a).astype(np.uint8)
    y = rng.integers(0, 4, b).astype(np.uint8)
    z = np.full(g, 4, dtype=np.uint8)
    expect = (a + b) * m - O - (g - 1) * X

    r = oracle.align(np.concatenate([x, y]), np.concatenate([x, z, y]), W, O, X)
    assert r["score1"] == expect
    assert (r["read_begin1"], r["ref_begin1"], r["read_end1"], r["ref_end1"]) == (0, 0, a + b - 1, a + b + g - 1)
    assert R.G(a + b - 1, expect) == g
    assert R.band(a + b, a + b + g, expect) == (0, g)
    assert check_pair(R, np.concatenate([x, y]), np.concatenate([x, z, y]))

    r = oracle.align(np.concatenate([x, z, y]), np.concatenate([x, y]), W, O, X)
    assert r["score1"] == expect
    assert R.Gn(a + b + g - 1, expect) == g
    assert R.band(a + b + g, a + b, expect) == (-g, 0)
    assert check_pair(R, np.concatenate([x, z, y]), np.concatenate([x, y]))


def test_band_widths_map_to_the_anti_diagonal_classes(lib):
    R = Rules(lib, dna(2, -3), 5, 2)
    seen = set()
    # targets longer than the rectangle's 4096 columns keep the band classes
    for s1 in range(20000, 200, -97):
        c, width = R.trace_class(5000, 5000, s1)
        expect = 0 if width <= 64 else 1 if width <= 128 else 2 if width <= 256 else 3 if width <= 512 else RING
        assert c == expect, (s1, width, c)
        seen.add(c)
    assert seen == {0, 1, 2, 3, RING}


def test_wide_bands_go_to_the_rectangle_when_it_fits(lib):
    rng = np.random.default_rng(5)
    # DNA: class 5 + min((la - 1) / 64, 3), for narrow bands too while the
    # rectangle costs at most 3x the band's anti-diagonal slots
    R = Rules(lib, dna(2, -3), 2, 1)
    for la in (40, 60, 100, 130, 200, 300, 600):
        c, width = R.trace_class(la, la + 50, 10)
        assert c == T16_FIRST + min((la - 1) // 64, 3), (la, width, c)
    c, width = R.trace_class(600, 650, 10)
    assert width > 512
    # DNA regions whose decisions exceed 2^17 words keep the ring kernel
    c, width = R.trace_class(1000, 1050, 10)
    assert width > 512 and c == RING
    assert lib.hr_t16_need_words(1000, 1050, 3) > (1 << 17)
    # general alphabet: 64-row strips, 128-row ones for regions whose
    # decisions exceed 2^17 words in 64-row strips (the large pair that the
    # routing once sent to the ring kernel by an overflow)
    P = Rules(lib, protein_like(rng), 11, 1)
    c, width = P.trace_class(1000, 1000, 50)
    assert width > 512 and c == T16_FIRST + 1
    assert lib.hr_t16_need_words(1000, 1000, 0) > (1 << 17)
    c, width = P.trace_class(500, 700, 50)
    assert width > 512 and c == T16_FIRST
    for la, lb in ((2000, 2100), (3000, 2500), (1200, 4096)):
        c, width = P.trace_class(la, lb, 30)
        assert width > 512 and c in (T16_FIRST, T16_FIRST + 1), (la, lb, c)
        assert lib.hr_t16_need_words(la, lb, c - T16_FIRST) <= (1 << 20)


def test_rectangle_refused_beyond_its_values_and_columns(lib):
    # a 600 x 650 region in 256-row strips: 768 rows, 666 columns padded
    la, lb = 600, 650
    # lowest value 3O + X(rows + cols + 2) + |wmin|: 28789 fits, 31672 does not
    c, width = Rules(lib, dna(44, -3), 22, 20).trace_class(la, lb, 10)
    assert width > 512 and c == T16_FIRST + 3
    c, width = Rules(lib, dna(44, -3), 22, 22).trace_class(la, lb, 10)
    assert width > 512 and c == RING
    # highest value wmax (min(rows, cols) + 1): 44 x 667 fits, 46 x 667 does not
    c, width = Rules(lib, dna(46, -3), 22, 20).trace_class(la, lb, 10)
    assert width > 512 and c == RING
    # columns: targets beyond 4096 letters
    R = Rules(lib, dna(2, -3), 3, 1)
    c, width = R.trace_class(60, 4096, 10)
    assert width > 512 and c == T16_FIRST
    c, width = R.trace_class(60, 4097, 10)
    assert width > 512 and c == RING


def test_routing_is_total_and_consistent_on_random_regions(lib):
    rng = np.random.default_rng(9)
    for it in range(3000):
        if rng.random() < 0.5:
            W, need_cap = dna(int(rng.integers(1, 6)), -int(rng.integers(1, 6))), 1 << 17
        else:
            W, need_cap = protein_like(rng), 1 << 20
        X = int(rng.integers(1, 5))
        R = Rules(lib, W, X + int(rng.integers(0, 12)), X)
        la = int(rng.integers(1, 6000))
        lb = int(rng.integers(1, 6000))
        s1 = int(rng.integers(1, 2 * int(W.max()) * min(la, lb) + 2))
        c, width = R.trace_class(la, lb, s1, small=bool(rng.random() < 0.5))
        assert 0 <= c <= T16_FIRST + 3
        if c >= T16_FIRST:
            assert lb <= 4096
            assert lib.hr_t16_need_words(la, lb, c - T16_FIRST) <= need_cap
            if W.shape[0] != 4:
                assert c in (T16_FIRST, T16_FIRST + 1)
        else:
            expect = 0 if width <= 64 else 1 if width <= 128 else 2 if width <= 256 else 3 if width <= 512 else RING
            assert c == expect


NEG = -(1 << 30)


def first_reversed_max(q, t, W, O, X, eq, et, score1, band=None):
    """Local Gotoh fill over reverse(q[0..eq]) x reverse(t[0..et]), written
    out cell by cell; with band = (Gn, G) the cells off the diagonals
    [-Gn, G] (j - i, reversed) are never computed: H = 0, E = F = -inf there,
    the fill kernel's boundary values.  Returns the first cell, by column and
    then row, whose H equals score1, as a begin (begin_q, begin_t)."""
    m, n = eq + 1, et + 1
    Hp = [0] * (n + 1)          # row i-1 of H, column 0 is the boundary
    Fp = [NEG] * (n + 1)
    Hrows = []
    for i in range(1, m + 1):
        a = int(q[eq - (i - 1)])
        H = [0] * (n + 1)
        F = [NEG] * (n + 1)
        E = NEG
        for j in range(1, n + 1):
            if band is not None and not (-band[0] <= (j - i) <= band[1]):
                H[j], F[j], E = 0, NEG, NEG
                continue
            E = max(H[j - 1] - O, E - X)
            F[j] = max(Hp[j] - O, Fp[j] - X)
            H[j] = max(0, Hp[j - 1] + int(W[a, int(t[et - (j - 1)])]), E, F[j])
        Hrows.append(H)
        Hp, Fp = H, F
    for j in range(1, n + 1):
        for i in range(1, m + 1):
            if Hrows[i - 1][j] == score1:
                return eq - (i - 1), et - (j - 1)
    return None


@pytest.mark.parametrize("kind", ["related", "one_gap"])
def test_banded_reversed_fill_finds_the_same_begin(lib, kind):
    """The reversed fill restricted to the reverse band [-Gn, G] reaches
    score1 first at the same cell as the unrestricted one, the oracle's begin:
    every path reaching score1 starts at the reversed origin and stays in the
    band, and a restriction only lowers the other cells."""
    rng = np.random.default_rng(21 if kind == "related" else 22)
    checked = narrow = tight = 0
    for it in range(40):
        if kind == "related":
            A = 4
            W = dna(int(rng.integers(1, 4)), -int(rng.integers(1, 5)))
            X = int(rng.integers(1, 4))
            O = X + int(rng.integers(0, 6))
            base = rng.integers(0, A, int(rng.integers(10, 70))).astype(np.uint8)
            q = mutate(rng, base, A, sub=0.1, indel=0.1, max_run=4)
            t = np.concatenate([rng.integers(0, A, int(rng.integers(0, 20))).astype(np.uint8),
                                mutate(rng, base, A, sub=0.05, indel=0.05, max_run=4),
                                rng.integers(0, A, int(rng.integers(0, 20))).astype(np.uint8)])
        else:
            A, O, X = 5, 5, 2
            W = dna(2, -3, A)
            g = int(rng.integers(1, 9))
            x = rng.integers(0, 4, int(rng.integers(g + 4, 40))).astype(np.uint8)
            y = rng.integers(0, 4, int(rng.integers(g + 4, 40))).astype(np.uint8)
            z = np.full(g, 4, np.uint8)
            q, t = (np.concatenate([x, y]), np.concatenate([x, z, y]))
            if it % 2:
                q, t = t, q
            t = np.concatenate([rng.integers(0, 4, int(rng.integers(0, 15))).astype(np.uint8), t])
        R = Rules(lib, W, O, X)
        r = oracle.align(q, t, R.W, O, X)
        s1 = r["score1"]
        if s1 <= 0:
            continue
        eq, et = r["read_end1"], r["ref_end1"]
        begin = (r["read_begin1"], r["ref_begin1"])
        G, Gn = R.G(eq, s1), R.Gn(eq, s1)
        assert first_reversed_max(q, t, R.W, O, X, eq, et, s1) == begin
        assert first_reversed_max(q, t, R.W, O, X, eq, et, s1, band=(Gn, G)) == begin
        checked += 1
        narrow += (G + Gn + 1) < min(eq + 1, et + 1)
        if kind == "one_gap" and G > 0 and Gn > 0:
            # the one-gap path touches an edge: one diagonal less loses the begin
            tight += (first_reversed_max(q, t, R.W, O, X, eq, et, s1, band=(Gn, G - 1)) != begin) + \
                (first_reversed_max(q, t, R.W, O, X, eq, et, s1, band=(Gn - 1, G)) != begin)
    assert checked >= 30 and narrow >= 10
    if kind == "one_gap":
        assert tight >= 15


def global_cigar(qs, ts, W, O, X, band=None):
    """Global Gotoh over qs x ts (a gap of k letters costs O + (k-1)X),
    written out cell by cell, and its traceback from the end in state H with
    the fixed preference: diagonal, then the E state (D, target letters),
    then F (I, query letters); in E and F an open is preferred to an extend.
    With band = (dlo, dhi) the cells off the diagonals [dlo, dhi] (j - i) are
    -inf.  Returns the CIGAR as (length, op) runs, op 0/1/2 = M/I/D, and the
    score; (None, None) when the band leaves out the end cell."""
    la, lb = len(qs), len(ts)
    H = [[NEG] * (lb + 1) for _ in range(la + 1)]
    E = [[NEG] * (lb + 1) for _ in range(la + 1)]
    F = [[NEG] * (lb + 1) for _ in range(la + 1)]
    inb = lambda i, j: band is None or band[0] <= j - i <= band[1]
    H[0][0] = 0
    for i in range(la + 1):
        for j in range(lb + 1):
            if (i == 0 and j == 0) or not inb(i, j):
                continue
            if j > 0:
                E[i][j] = max(H[i][j - 1] - O, E[i][j - 1] - X)
            if i > 0:
                F[i][j] = max(H[i - 1][j] - O, F[i - 1][j] - X)
            d = H[i - 1][j - 1] + int(W[int(qs[i - 1]), int(ts[j - 1])]) if i > 0 and j > 0 else NEG
            H[i][j] = max(d, E[i][j], F[i][j])
    if H[la][lb] <= NEG // 2:
        return None, None
    ops = []
    i, j, state = la, lb, 0
    while i > 0 or j > 0:
        if state == 0:
            if i > 0 and j > 0 and H[i][j] == H[i - 1][j - 1] + int(W[int(qs[i - 1]), int(ts[j - 1])]):
                ops.append(0)
                i, j = i - 1, j - 1
                continue
            state = 1 if H[i][j] == E[i][j] else 2
        if state == 1:
            ops.append(2)
            state = 0 if E[i][j] == H[i][j - 1] - O else 1
            j -= 1
        else:
            ops.append(1)
            state = 0 if F[i][j] == H[i - 1][j] - O else 2
            i -= 1
    runs = []
    for op in reversed(ops):
        if runs and runs[-1][1] == op:
            runs[-1] = (runs[-1][0] + 1, op)
        else:
            runs.append((1, op))
    return runs, H[la][lb]


@pytest.mark.parametrize("kind", ["related", "two_gaps"])
def test_banded_traceback_gives_the_full_rectangle_cigar(lib, kind):
    """Global alignment between begin and end on the band [dlo, dhi] gives
    the oracle's canonical CIGAR (full rectangle): optimal paths lie in the
    band, so their cells keep their values and every preference test decides
    alike.  Two-gap pairs (x + z1 + y against x + z2 + y, z1 and z2 g letters
    that mismatch at -20, so both are gapped out) have begin and end on
    diagonal 0 and a path reaching diagonal g or -g; the score bound gives
    the band [-g, g] exactly, and one diagonal less on the path's side loses
    the CIGAR."""
    rng = np.random.default_rng(31 if kind == "related" else 32)
    checked = tight = 0
    for it in range(40):
        if kind == "related":
            A = 4
            W = dna(int(rng.integers(1, 4)), -int(rng.integers(1, 5)))
            X = int(rng.integers(1, 4))
            O = X + int(rng.integers(0, 6))
            base = rng.integers(0, A, int(rng.integers(10, 60))).astype(np.uint8)
            q = mutate(rng, base, A, sub=0.1, indel=0.1, max_run=4)
            t = mutate(rng, base, A, sub=0.05, indel=0.05, max_run=4)
        else:
            A, O, X = 6, 5, 2
            W = dna(2, -3, A)
            W[4, 5] = W[5, 4] = -20
            g = int(rng.integers(1, 7))
            x = rng.integers(0, 4, int(rng.integers(2 * g + 8, 40))).astype(np.uint8)
            y = rng.integers(0, 4, int(rng.integers(2 * g + 8, 40))).astype(np.uint8)
            q = np.concatenate([x, np.full(g, 4, np.uint8), y])
            t = np.concatenate([x, np.full(g, 5, np.uint8), y])
        R = Rules(lib, W, O, X)
        r = oracle.align(q, t, R.W, O, X)
        s1 = r["score1"]
        if s1 <= 0:
            continue
        qs = q[r["read_begin1"]: r["read_end1"] + 1]
        ts = t[r["ref_begin1"]: r["ref_end1"] + 1]
        dlo, dhi = R.band(len(qs), len(ts), s1)
        full, sc_full = global_cigar(qs, ts, R.W, O, X)
        banded, sc_band = global_cigar(qs, ts, R.W, O, X, band=(dlo, dhi))
        assert sc_full == s1 and sc_band == s1
        assert full == r["cigar"] and banded == r["cigar"]
        checked += 1
        if kind == "two_gaps":
            assert s1 == 2 * (len(x) + len(y)) - 2 * (O + (g - 1) * X)
            assert (dlo, dhi) == (-g, g)
            lost = [global_cigar(qs, ts, R.W, O, X, band=cut)[0] != r["cigar"]
                    for cut in ((dlo + 1, dhi), (dlo, dhi - 1))]
            tight += any(lost)
    assert checked >= 30
    if kind == "two_gaps":
        assert tight == checked


def test_batch_status_precedence(lib):
    """A batch's return code from its kernels' counts: bad letters, then
    records flagged by a consistency check, then CIGAR space (with GSW_CIGAR
    only); otherwise GSW_OK."""
    from paper_1208_6350_gb300 import gsw
    st = lib.hr_batch_status
    assert st(0, 0, 1, 10, 10) == gsw.GSW_OK
    assert st(0, 0, 1, 11, 10) == gsw.GSW_ECIGAR_SPACE
    assert st(0, 0, 0, 11, 10) == gsw.GSW_OK          # no CIGAR asked: words never counted
    assert st(0, 0, 1, 1, 0) == gsw.GSW_ECIGAR_SPACE
    assert st(0, 1, 1, 11, 10) == gsw.GSW_EINTERNAL   # one flagged record is loud
    assert st(0, 5, 0, 0, 0) == gsw.GSW_EINTERNAL
    assert st(1, 5, 1, 11, 10) == gsw.GSW_EINVAL      # bad input first
    assert st(1, 0, 0, 0, 0) == gsw.GSW_EINVAL


def test_fill_launch_mask_holds_every_class_the_plan_can_pick(lib):
    """Each fill launch leaves out the classes outside a mask computed on the
    host from the longest query: every class the plan picks for a query of at
    most that many rows (forward; reverse with and without 32-bit pairs; any
    tune table, including the CTA class for short buckets) is in the mask, and
    a short-read batch under a one-class table launches few classes."""
    rng = np.random.default_rng(77)
    codes = [-1, 0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13]
    for A, W in ((4, dna(2, -3)), (20, protein_like(rng))):
        Wc = np.ascontiguousarray(W.astype(np.int8))
        Wp = Wc.ctypes.data_as(ctypes.c_void_p)
        for trial in range(40):
            table = np.full(32, -1, np.int8)
            if trial % 4:
                table[:] = rng.choice(codes, 32)
            tp = table.ctypes.data_as(ctypes.c_void_p)
            maxm = int(rng.choice([1, 31, 100, 250, 1024, 1025, 1800, 5000, 30000]))
            for mode in (0, 2):
                for s32 in (0, 1):
                    if mode == 0 and s32:
                        continue
                    mask = lib.hr_fill_class_mask(A, Wp, 5, 2, tp, mode, maxm, 0, s32)
                    rows = set(rng.integers(1, maxm + 1, 300).tolist()) | {1, maxm}
                    for r in rows:
                        for s in ((0, 1) if s32 else (0,)):
                            c = lib.hr_pick_class(A, Wp, 5, 2, tp, mode, int(r), s)
                            assert (mask >> c) & 1, (A, mode, maxm, r, s, c, bin(mask))
                    if mode == 0:
                        assert mask & 1  # empty pairs take class 0
    # the short-read case: every bucket of up to 250 rows tuned to the 8-lane
    # variants (public codes 9..13): the forward launch holds those and class 0
    W = np.ascontiguousarray(dna(2, -2).astype(np.int8))
    table = np.full(32, -1, np.int8)
    table[:8] = [9, 9, 9, 9, 10, 11, 12, 13]
    m = lib.hr_fill_class_mask(4, W.ctypes.data_as(ctypes.c_void_p), 3, 1, table.ctypes.data_as(ctypes.c_void_p),
                               0, 250, 0, 0)
    assert bin(m).count("1") == 6
