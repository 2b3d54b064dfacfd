"""GPU parity: every output of the CUDA path equals the oracle's, element by
element (integers: zero tolerance), on seeded inputs shaped like the paper's
workloads, at sizes that span several fill variants, strips and a ragged
tail, plus constructed edge cases (empty and length-1 sequences, no shared
letters, exact ties, 16-bit overflow threshold, multi-strip queries)."""
import numpy as np
import pytest

from paper_1208_6350_gb300 import gsw, workloads as wl
from parity_util import compare, run_gpu_device, run_gpu_host, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gsw.Context(0, 8 << 30)
    yield c
    c.close()


def mixed_dna(seed, npairs, qmax, tmax, match=2, mismatch=-2, O=3, X=1, related=0.7):
    """Ragged DNA pairs: lengths from 0 to the maxima, many with an implanted
    mutated copy of the query."""
    rng = np.random.default_rng(seed)
    ql = rng.integers(0, qmax + 1, npairs)
    tl = rng.integers(0, tmax + 1, npairs)
    ql[:4] = [0, 1, 0, 1]
    tl[:4] = [0, 0, 1, 1]
    qs = [rng.integers(0, 4, n).astype(np.uint8) for n in ql]
    ts = []
    for p in range(npairs):
        t = rng.integers(0, 4, tl[p]).astype(np.uint8)
        if rng.random() < related and len(qs[p]) and len(t) >= len(qs[p]):
            cp = qs[p].copy()
            mut = rng.random(len(cp)) < 0.05
            cp[mut] = rng.integers(0, 4, int(mut.sum()))
            o = int(rng.integers(0, len(t) - len(cp) + 1))
            t[o:o + len(cp)] = cp
        ts.append(t)
    return _batch(qs, ts, wl.dna_matrix(match, mismatch), O, X, "mixed")


def _batch(qs, ts, W, O, X, name, alphabet="ACGT"):
    ql = np.array([len(x) for x in qs], np.int32)
    tl = np.array([len(x) for x in ts], np.int32)
    qo = np.concatenate([[0], np.cumsum(ql)[:-1]]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(tl)[:-1]]).astype(np.int64)
    q = np.concatenate(qs + [np.zeros(0, np.uint8)]).astype(np.uint8)
    t = np.concatenate(ts + [np.zeros(0, np.uint8)]).astype(np.uint8)
    return wl.Batch(name, q, qo, ql, t, to, tl, W, O, X, alphabet)


def test_mixed_small_all_outputs_host_io(ctx):
    b = mixed_dna(1, 400, 300, 700)
    compare(b, run_oracle(b), run_gpu_host(ctx, b))


def test_mixed_small_device_path(ctx):
    b = mixed_dna(2, 300, 260, 500)
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_config1_subset(ctx):
    b = wl.config1().subset(np.arange(0, 1000, 4))
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_config2_sample_with_decoys(ctx):
    b = wl.config2(4000, seed=11)
    idx = np.random.default_rng(0).permutation(b.npairs)[:1500]
    s = b.subset(idx)
    assert s.meta["decoy"].any()
    compare(s, run_oracle(s), run_gpu_device(ctx, s))


def test_forced_32bit_lanes(ctx):
    b = mixed_dna(3, 200, 300, 600)
    got = run_gpu_host(ctx, b, flags=gsw.GSW_CIGAR | gsw.GSW_FORCE_S32)
    assert (got[0]["flags"] & gsw.GSW_RES_S32).all()
    compare(b, run_oracle(b), got)


def test_score_only_and_begin_only(ctx):
    b = mixed_dna(4, 200, 200, 400)
    ora = run_oracle(b)
    got = run_gpu_host(ctx, b, flags=0)
    compare(b, ora, got, check_begin=False, check_cigar=False)
    assert (got[0]["ref_begin1"] == -1).all() and (got[0]["cigar_len"] == 0).all()
    got = run_gpu_host(ctx, b, flags=gsw.GSW_BEGIN)
    compare(b, ora, got, check_cigar=False)


@pytest.mark.parametrize("mask_len", [0, 5, 40, 1000])
def test_mask_lengths(ctx, mask_len):
    b = mixed_dna(5, 150, 120, 600)
    compare(b, run_oracle(b, mask_len), run_gpu_host(ctx, b, mask_len=mask_len))


def test_sixteen_bit_overflow_threshold(ctx):
    # match 100: a self-alignment of length L scores 100 L; 16-bit lanes are
    # exact up to 32767 - 100 = 32667, so L = 326 stays in 16 bits and
    # L = 327 must be refilled in 32-bit lanes.
    rng = np.random.default_rng(6)
    W = wl.dna_matrix(100, -100)
    qs, ts = [], []
    for L in (325, 326, 327, 328, 400):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q)
        ts.append(np.concatenate([rng.integers(0, 4, 50), q, rng.integers(0, 4, 30)]).astype(np.uint8))
    b = _batch(qs, ts, W, 30, 10, "overflow")
    got = run_gpu_host(ctx, b)
    s32 = (got[0]["flags"] & gsw.GSW_RES_S32) != 0
    assert list(s32) == [False, False, True, True, True]
    compare(b, run_oracle(b), got)


def test_multi_strip_long_queries(ctx):
    b = wl.dna_long_reads(12, 600, 2500, seed=7)
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_protein_general_matrix(ctx):
    ps = wl.protein_search(20, 200, seed=8)
    rng = np.random.default_rng(9)
    qi = rng.integers(0, 20, 300)
    di = rng.integers(0, 200, 300)
    qi[:10] = ps.queries.meta["homolog_query"][:10]
    di[:10] = ps.queries.meta["homolog_db"][:10]
    b = ps.pairs(qi, di).subset(np.arange(300))
    compare(b, run_oracle(b), run_gpu_host(ctx, b))


def test_small_alphabet_and_odd_scoring(ctx):
    rng = np.random.default_rng(10)
    A = 3
    W = rng.integers(-3, 4, (A, A)).astype(np.int8)
    W[0, 0] = 3
    qs = [rng.integers(0, A, int(n)).astype(np.uint8) for n in rng.integers(0, 90, 120)]
    ts = [rng.integers(0, A, int(n)).astype(np.uint8) for n in rng.integers(0, 200, 120)]
    for O, X in ((2, 2), (5, 1), (0, 0), (4, 0)):
        b = _batch(qs, ts, W, O, X, "odd", "ACG")
        compare(b, run_oracle(b), run_gpu_host(ctx, b))


def test_profile_api_matches_batch(ctx):
    rng = np.random.default_rng(12)
    W = wl.dna_matrix(2, -3)
    q = rng.integers(0, 4, 150).astype(np.uint8)
    ts = []
    for k in range(64):
        t = rng.integers(0, 4, int(rng.integers(100, 900))).astype(np.uint8)
        if k % 2 and len(t) > 160:
            o = int(rng.integers(0, len(t) - 150))
            t[o:o + 150] = q
        ts.append(t)
    b = _batch([q] * 64, ts, W, 5, 2, "profile")
    prof = gsw.gsw_profile_create(ctx.handle, q, W, 5, 2)
    try:
        res = np.zeros(64, gsw.RESULT_DTYPE)
        cap = 64 * 200
        cig = np.zeros(cap, np.uint32)
        gsw.gsw_align_profile(ctx.handle, prof, 64, b.t, b.t_off, b.t_len,
                              gsw.GSW_CIGAR | gsw.GSW_HOST_IO, -1, res, cig, cap)
    finally:
        gsw.gsw_profile_destroy(prof)
    compare(b, run_oracle(b), (res, cig, (None, None)), check_colmax=False)


def test_cigar_space_error_reported(ctx):
    b = mixed_dna(13, 50, 100, 200, related=1.0)
    res, cig, _, rc = ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, 3, 1,
                                     gsw.GSW_CIGAR, -1, cigar_capacity=3)
    assert rc == gsw.GSW_ECIGAR_SPACE
    assert (res["flags"] & gsw.GSW_RES_CIGAR_SPACE).any()


def test_invalid_letter_rejected(ctx):
    b = mixed_dna(14, 10, 50, 60)
    b.t[b.t_off[5]] = 7  # not in the 4-letter alphabet
    with pytest.raises(gsw.GswError) as ei:
        ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, 3, 1)
    assert ei.value.code == gsw.GSW_EINVAL


def test_plain_per_pair_baseline_matches(ctx):
    b = mixed_dna(15, 40, 120, 300)
    got = run_gpu_host(ctx, b, flags=gsw.GSW_CIGAR | gsw.GSW_PLAIN)
    compare(b, run_oracle(b), got)


def test_long_reads_wide_bands(ctx):
    # 10 % error reads of 3-6 kb: bands of several hundred to a few thousand
    # diagonals (wide anti-diagonal traceback), queries of 12-24 strips
    b = wl.dna_long_reads(5, 3000, 6000, seed=17)
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def _implanted(rng, A, qlens, flank, p_sub):
    """Random queries over A letters, each implanted with substitutions into a
    random target `flank` times its length."""
    qs, ts = [], []
    for L in qlens:
        q = rng.integers(0, A, int(L)).astype(np.uint8)
        cp = q.copy()
        mut = rng.random(len(cp)) < p_sub
        cp[mut] = rng.integers(0, A, int(mut.sum()))
        t = rng.integers(0, A, int(flank * L)).astype(np.uint8)
        o = int(rng.integers(0, len(t) - len(cp) + 1))
        t[o:o + len(cp)] = cp
        qs.append(q)
        ts.append(t)
    return qs, ts


def test_cta_kernel_many_strips(ctx):
    # queries of 1,800-9,000 rows (up to 9 strips of 1,024 rows, ragged last
    # strips): the CTA kernel, with more strips than its 4 warps and several
    # pairs in flight per CTA, mixed in one batch with short pairs of the
    # per-group variants
    lb = wl.dna_long_reads(10, 1800, 9000, seed=21)
    sb = mixed_dna(22, 60, 300, 900)
    b = wl.concat([lb, wl.Batch(sb.name, sb.q, sb.q_off, sb.q_len, sb.t, sb.t_off, sb.t_len, lb.W,
                                lb.gap_open, lb.gap_extend, "ACGT")])
    assert (b.q_len > 1792).sum() >= 8
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_cta_kernel_32bit_lanes(ctx):
    # forced 32-bit lanes: the 32-bit CTA class (256 rows per strip)
    b = wl.dna_long_reads(4, 1000, 2600, seed=23)
    got = run_gpu_host(ctx, b, flags=gsw.GSW_CIGAR | gsw.GSW_FORCE_S32)
    assert (got[0]["flags"] & gsw.GSW_RES_S32).all()
    compare(b, run_oracle(b), got)


def test_cta_kernel_overflow_rerun(ctx):
    # match 20: 2-3 kb near-identical alignments score ~40000-60000, past the
    # 16-bit bound, so the 16-bit CTA fill flags them and the 32-bit CTA
    # fill redoes them
    rng = np.random.default_rng(24)
    qs, ts = _implanted(rng, 4, [2000, 2400, 3000], 1.2, 0.02)
    b = _batch(qs, ts, wl.dna_matrix(20, -20), 30, 10, "overflow-long")
    got = run_gpu_host(ctx, b)
    assert (got[0]["flags"] & gsw.GSW_RES_S32).all()
    compare(b, run_oracle(b), got)


def test_cta_kernel_general_alphabet(ctx):
    # a 20-letter matrix with queries of more than 8 strips (general-alphabet
    # CTA kernel) beside short ones
    rng = np.random.default_rng(25)
    qs, ts = _implanted(rng, 20, [4200, 4700, 300, 150], 1.1, 0.3)
    b = _batch(qs, ts, wl.synthetic_protein_matrix(), 11, 1, "protein-long",
               "ARNDCQEGHILKMFPSTWYV")
    compare(b, run_oracle(b), run_gpu_host(ctx, b))


def _indel_pairs(rng, specs, p_sub=0.05):
    """Queries from a random source with one inserted block and/or one deleted
    block (bands clipped by either end of the alignment), targets = random
    flanks + the source."""
    qs, ts = [], []
    for L, ins, dele in specs:
        s = rng.integers(0, 4, L).astype(np.uint8)
        q = np.concatenate([s[: L // 3], rng.integers(0, 4, ins).astype(np.uint8), s[L // 3:]])
        if dele:
            c = 2 * len(q) // 3
            q = np.concatenate([q[:c], q[c + dele:]])
        mut = rng.random(len(q)) < p_sub
        q[mut] = rng.integers(0, 4, int(mut.sum()))
        t = np.concatenate([rng.integers(0, 4, 200), s, rng.integers(0, 4, 150)]).astype(np.uint8)
        qs.append(q)
        ts.append(t)
    return qs, ts


@pytest.mark.parametrize("O,X", [(4, 2), (3, 3), (5, 0)])
def test_wide_band_traceback_indels_and_gap_costs(ctx, O, X):
    # bands of 600 to all diagonals (extend 0: every diagonal) through the CTA
    # strip traceback: a 300-letter insertion, a 300-letter deletion, both,
    # and open == extend (the open bit of every gap cell)
    rng = np.random.default_rng(31 + O + X)
    qs, ts = _indel_pairs(rng, [(2500, 300, 0), (2500, 0, 300), (3000, 150, 150), (1800, 0, 0)])
    b = _batch(qs, ts, wl.dna_matrix(2, -4), O, X, "indels")
    compare(b, run_oracle(b), run_gpu_host(ctx, b))


@pytest.mark.parametrize("seed", [40, 41, 42, 44])
def test_any_fill_class_table_gives_the_same_results(ctx, seed):
    # the autotuner may give any query length any class: per-group variants
    # with one or several strips, or the CTA kernel; forward and reversed
    # fills must stay exact under each
    rng = np.random.default_rng(seed)
    table = [int(rng.choice([0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13])) for _ in range(gsw.TUNE_BUCKETS)]
    b = mixed_dna(seed, 160, 1024, 1400)
    ora = run_oracle(b)
    ctx.set_tune(table)
    try:
        compare(b, ora, run_gpu_device(ctx, b))
    finally:
        ctx.set_tune(None)


def test_autotune_table_is_valid_and_exact():
    c = gsw.Context(0, 4 << 30)
    try:
        W = wl.dna_matrix(2, -2)
        t = c.autotune(W, 3, 1, target_len=600)
        assert len(t["fill_class"]) == gsw.TUNE_BUCKETS
        assert all(x in (0, 1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 12, 13) for x in t["fill_class"])
        assert all(g > 0 for g in t["gcups"]) and all(g >= d for g, d in zip(t["gcups"], t["gcups_default"]))
        b = mixed_dna(43, 200, 900, 1200)
        compare(b, run_oracle(b), run_gpu_host(c, b))
    finally:
        c.close()


def test_repeated_call_replays_captured_graphs(ctx):
    # the same buffers, sizes and flags on a stream of its own: eager, eager
    # (first capture key), captured, then replayed; new letters in the same
    # buffers are read by the replay; results equal the oracle's every time
    import torch
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(dev)
    b = mixed_dna(50, 300, 260, 700)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, t = T(b.q), T(b.t)
    qo, to = T(b.q_off.astype(np.int64)), T(b.t_off.astype(np.int64))
    ql, tl = T(b.q_len.astype(np.int32)), T(b.t_len.astype(np.int32))
    n = b.npairs
    res = torch.zeros(n * 12, dtype=torch.int32, device=dev)
    cap = int(b.q_len.sum() + b.t_len.sum() + 16)
    cig = torch.zeros(cap, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def call():
        rc = gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, b.W, b.gap_open, b.gap_extend,
                                 gsw.GSW_CIGAR, -1, res, cig, cap, stream=s)
        torch.cuda.synchronize()
        assert rc == gsw.GSW_OK
        return (res.cpu().numpy().view(gsw.RESULT_DTYPE).copy(), cig.cpu().numpy().view(np.uint32).copy(),
                (None, None)), gsw.gsw_last_stats(ctx.handle)["graph_segments"]

    ora = run_oracle(b, colmax=False)
    segs = []
    for _ in range(5):
        got, g = call()
        compare(b, ora, got, check_colmax=False)
        segs.append(g)
    assert segs[-1] == 2 and segs[0] == 0
    # new letters, same lengths: the replayed graph reads them
    rng = np.random.default_rng(51)
    b2 = wl.Batch(b.name, rng.integers(0, 4, len(b.q)).astype(np.uint8), b.q_off, b.q_len, b.t.copy(),
                  b.t_off, b.t_len, b.W, b.gap_open, b.gap_extend, b.alphabet)
    b2.t[: len(b2.t) // 2] = rng.integers(0, 4, len(b2.t) // 2)
    q.copy_(T(b2.q))
    t.copy_(T(b2.t))
    torch.cuda.synchronize()
    got, g = call()
    assert g >= 1  # the first segment replays; the second depends on the new traceback needs
    compare(b2, run_oracle(b2, colmax=False), got, check_colmax=False)


def test_large_batch_uses_the_band_kernel(ctx):
    # from 2^14 pairs on, narrow bands go to the thread-per-pair band kernel
    # (reverse + traceback in one thread); smaller batches take the warp
    # kernels.  Every pair of a 20,000-pair short-read batch is compared.
    b = wl.config2(20000, seed=12)
    assert b.npairs >= 1 << 14
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_empty_batch_and_all_empty_pairs(ctx):
    # zero pairs is a no-op; pairs with an empty query or target give score
    # 0, positions -1 and no CIGAR (the oracle's empty alignment)
    res, cig, _, rc = ctx.align_host(np.zeros(0, np.uint8), np.zeros(0, np.int64), np.zeros(0, np.int32),
                                     np.zeros(0, np.uint8), np.zeros(0, np.int64), np.zeros(0, np.int32),
                                     wl.dna_matrix(2, -2), 3, 1)
    assert rc == gsw.GSW_OK and len(res) == 0
    qs = [np.zeros(0, np.uint8), np.array([1, 2], np.uint8), np.zeros(0, np.uint8)]
    ts = [np.array([0, 1, 2], np.uint8), np.zeros(0, np.uint8), np.zeros(0, np.uint8)]
    b = _batch(qs, ts, wl.dna_matrix(2, -2), 3, 1, "empty")
    got = run_gpu_host(ctx, b)
    compare(b, run_oracle(b), got)
    assert (got[0]["score1"] == 0).all() and (got[0]["cigar_len"] == 0).all()
    assert (got[0]["ref_end1"] == -1).all() and (got[0]["read_begin1"] == -1).all()


@pytest.mark.parametrize("host_io", [True, False])
def test_packed_2bit_inputs(ctx, host_io):
    # GSW_PACKED2: both arenas 4 letters to a byte, offsets in letters (not
    # multiples of 4), expanded on the device; results equal the oracle's on
    # the unpacked letters
    b = mixed_dna(60, 300, 260, 700)
    ora = run_oracle(b)
    qp, tp = gsw.pack2(b.q), gsw.pack2(b.t)
    packed = wl.Batch(b.name, qp, b.q_off, b.q_len, tp, b.t_off, b.t_len, b.W, b.gap_open, b.gap_extend,
                      b.alphabet)
    flags = gsw.GSW_CIGAR | gsw.GSW_PACKED2
    got = run_gpu_host(ctx, packed, flags=flags) if host_io else run_gpu_device(ctx, packed, flags=flags)
    compare(b, ora, got)


def _weak_pairs(rng, lens, ident=0.75, p_indel=0.02, flank=(0, 120), A=4):
    """Query of each length, target = flanks + a copy at `ident` identity with
    scattered 1-3 letter indels: the local alignment spans about the whole
    query with a low score, so the provable band covers most of the region."""
    qs, ts = [], []
    for L in lens:
        q = rng.integers(0, A, L).astype(np.uint8)
        c = []
        for x in q:
            u = rng.random()
            if u < p_indel / 2:
                continue
            if u < p_indel:
                c.extend(rng.integers(0, A, int(rng.integers(1, 4))).tolist())
            c.append(int(x) if rng.random() < ident else int(rng.integers(0, A)))
        left, right = (int(rng.integers(flank[0], flank[1] + 1)) for _ in range(2))
        t = np.concatenate([rng.integers(0, A, left), np.array(c, np.int64), rng.integers(0, A, right)])
        qs.append(q)
        ts.append(t.astype(np.uint8))
    return qs, ts


@pytest.mark.parametrize("O,X", [(3, 1), (2, 2), (6, 0)])
def test_rect16_traceback_region_classes(ctx, O, X):
    # weak similarities whose regions fall on both sides of every row class of
    # the 16-bit rectangle traceback (64/128/192/256 rows) and up to its
    # 1024-column limit; open == extend and extend 0 exercise the tie rules
    rng = np.random.default_rng(70 + O * 10 + X)
    lens = [1, 2, 15, 40, 63, 64, 65, 100, 127, 128, 129, 160, 191, 192, 193, 230, 255, 256, 257, 300]
    qs, ts = _weak_pairs(rng, lens * 3)
    q2, t2 = _weak_pairs(rng, [200, 240, 256], flank=(700, 760))  # targets near 1,024 letters
    b = _batch(qs + q2, ts + t2, wl.dna_matrix(2, -2), O, X, "weak")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_rect16_traceback_general_alphabet(ctx):
    # a 20-letter alphabet with a BLOSUM-like matrix: regions up to 128 rows
    # take the 16-bit rectangle (one score table per lane)
    rng = np.random.default_rng(77)
    A = 20
    M = rng.integers(-4, 3, (A, A))
    M = ((M + M.T) // 2).astype(np.int8)
    np.fill_diagonal(M, rng.integers(4, 12, A))
    qs, ts = _weak_pairs(rng, [10, 50, 64, 65, 90, 127, 128, 129, 150] * 4, ident=0.6, A=A)
    b = _batch(qs, ts, M, 11, 1, "weak_protein", alphabet="ARNDCQEGHILKMFPSTWYV")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


@pytest.mark.parametrize("O,X", [(3, 1), (2, 2), (5, 0)])
def test_rect16_traceback_several_strips(ctx, O, X):
    # regions taller than one strip (256 rows for DNA) run strip after strip
    # with the boundary row in scratch; rows on both sides of each strip edge
    rng = np.random.default_rng(80 + O * 10 + X)
    qs, ts = _weak_pairs(rng, [257, 300, 383, 511, 512, 513, 600, 700, 767, 768, 769] * 2, flank=(0, 300))
    b = _batch(qs, ts, wl.dna_matrix(2, -2), O, X, "weak_strips")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_rect16_traceback_general_alphabet_strips(ctx):
    # 128-row strips for a 20-letter alphabet: regions of 1-4 strips
    rng = np.random.default_rng(81)
    A = 20
    M = rng.integers(-4, 3, (A, A))
    M = ((M + M.T) // 2).astype(np.int8)
    np.fill_diagonal(M, rng.integers(4, 12, A))
    qs, ts = _weak_pairs(rng, [129, 200, 255, 256, 257, 383, 384, 385, 500] * 2, ident=0.6, A=A)
    b = _batch(qs, ts, M, 11, 1, "weak_protein_strips", alphabet="ARNDCQEGHILKMFPSTWYV")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_protein_search_sample(ctx):
    # random query x database pairs of the protein search workload: long,
    # low-scoring local alignments with bands of hundreds of diagonals
    ps = wl.protein_search(n_queries=200, n_db=400, seed=9)
    rng = np.random.default_rng(9)
    b = ps.pairs(rng.integers(0, 200, 300), rng.integers(0, 400, 300))
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_reverse_band_edges_in_the_band_kernel(ctx):
    # 17,000 pairs (the thread-per-pair band kernel takes batches from 2^14):
    # reads with a run of 1-4 inserted (or deleted) letters a few letters
    # from their start end the reversed path below (or above) the main
    # diagonal, up to the reverse band's bounds on each side
    rng = np.random.default_rng(91)
    qs, ts = [], []
    for p in range(17000):
        L = int(rng.integers(60, 220))
        s = rng.integers(0, 4, L).astype(np.uint8)
        at = int(rng.integers(1, 12))
        k = int(rng.integers(1, 5))
        if p % 2:
            q = np.concatenate([s[:at], rng.integers(0, 4, k).astype(np.uint8), s[at:]])
        else:
            q = np.concatenate([s[:at], s[at + k:]])
        nsub = int(rng.integers(0, 3))
        if nsub:
            pos = rng.integers(0, len(q), nsub)
            q[pos] = (q[pos] + rng.integers(1, 4, nsub)) % 4
        t = np.concatenate([rng.integers(0, 4, int(rng.integers(0, 60))), s,
                            rng.integers(0, 4, int(rng.integers(0, 60)))]).astype(np.uint8)
        qs.append(q.astype(np.uint8))
        ts.append(t)
    b = _batch(qs, ts, wl.dna_matrix(2, -2), 3, 1, "edge_indels")
    assert b.npairs >= 1 << 14
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_band_kernels_mixed_widths_general_dna_matrix(ctx):
    # 17,000 pairs with a non-uniform 4x4 matrix (transitions -1, transversions
    # -3): the one-pair-per-thread band classes, with traceback bands of
    # several widths in one warp (reads with 0-8 substitutions and 0-2 indels
    # of 1-6 letters)
    rng = np.random.default_rng(93)
    M = np.full((4, 4), -3, np.int8)
    np.fill_diagonal(M, 2)
    for a, b_ in ((0, 2), (1, 3)):
        M[a, b_] = M[b_, a] = -1
    qs, ts = [], []
    for p in range(17000):
        L = int(rng.integers(80, 200))
        src = rng.integers(0, 4, L).astype(np.uint8)
        q = src.copy()
        for _ in range(int(rng.integers(0, 3))):
            at = int(rng.integers(5, len(q) - 5))
            k = int(rng.integers(1, 7))
            q = np.concatenate([q[:at], rng.integers(0, 4, k).astype(np.uint8), q[at:]]) if rng.random() < 0.5 \
                else np.concatenate([q[:at], q[at + k:]])
        nsub = int(rng.integers(0, 9))
        if nsub:
            pos = rng.integers(0, len(q), nsub)
            q[pos] = (q[pos] + rng.integers(1, 4, nsub)) % 4
        t = np.concatenate([rng.integers(0, 4, int(rng.integers(0, 80))), src,
                            rng.integers(0, 4, int(rng.integers(0, 80)))]).astype(np.uint8)
        qs.append(q.astype(np.uint8))
        ts.append(t)
    b = _batch(qs, ts, M, 4, 1, "mixed_widths_matrix")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_capped_fill_scratch_with_four_pairs_per_warp():
    # targets of 20,000 columns take 400 KB of column maxima and boundaries
    # per pair in flight, so a 512 MB budget caps the fill's scratch far below
    # the slots of a full launch; the 8-lane variants hold 4 pairs per warp,
    # and every launch stays within the slots the cap left (1,200 pairs, more
    # than the slots, so warps reuse theirs)
    rng = np.random.default_rng(161)
    qs, ts = [], []
    for L in rng.integers(120, 201, 1200):
        q = rng.integers(0, 4, int(L)).astype(np.uint8)
        c = q.copy()
        mut = rng.random(len(c)) < 0.03
        c[mut] = rng.integers(0, 4, int(mut.sum()))
        t = rng.integers(0, 4, 20000).astype(np.uint8)
        o = int(rng.integers(0, len(t) - len(c) + 1))
        t[o:o + len(c)] = c
        qs.append(q)
        ts.append(t)
    b = _batch(qs, ts, wl.dna_matrix(2, -3), 5, 2, "capped_scratch")
    small = gsw.Context(0, 512 << 20)
    try:
        got = run_gpu_device(small, b)
    finally:
        small.close()
    compare(b, run_oracle(b), got)


def test_band_kernel_cigars_of_many_runs(ctx):
    # 16,500 reads with 6-12 single-letter indels (alternately inserted and
    # deleted, at least 8 letters apart) under gap costs of 6 per letter:
    # narrow bands (the band kernel's traceback), CIGARs of 13-25 runs.  The
    # band kernel's walk keeps 16 runs and walks a longer CIGAR a second time
    # into its reserved words, so both kinds are here.
    rng = np.random.default_rng(151)
    qs, ts = [], []
    for p in range(16500):
        L = int(rng.integers(150, 221))
        src = rng.integers(0, 4, L).astype(np.uint8)
        k = int(rng.integers(6, 13))
        at = np.sort(rng.choice(np.arange(10, L - 10, 9), size=k, replace=False))
        q, last = [], 0
        for n, a in enumerate(at):
            q.append(src[last:a])
            if n % 2 == 0:
                q.append(rng.integers(0, 4, 1).astype(np.uint8))  # inserted letter
                last = a
            else:
                last = a + 1                                     # deleted letter
        q.append(src[last:])
        t = np.concatenate([rng.integers(0, 4, int(rng.integers(0, 50))), src,
                            rng.integers(0, 4, int(rng.integers(0, 50)))]).astype(np.uint8)
        qs.append(np.concatenate(q).astype(np.uint8))
        ts.append(t)
    b = _batch(qs, ts, wl.dna_matrix(2, -6), 6, 6, "many_runs")
    assert b.npairs >= 1 << 14
    ora = run_oracle(b)
    runs = ora[0]["cigar_len"]
    assert (runs > 16).sum() >= 1000 and ((runs > 1) & (runs <= 16)).sum() >= 1000
    compare(b, ora, run_gpu_device(ctx, b))


def test_rect16_traceback_large_regions_general_alphabet(ctx):
    # regions over a million cells (here 1,100-1,500 letters a side) exceed the
    # 64-row classes' per-pair words and take the 128-row class with its
    # larger allowance, in a launch of their own
    rng = np.random.default_rng(95)
    A = 20
    M = rng.integers(-4, 3, (A, A))
    M = ((M + M.T) // 2).astype(np.int8)
    np.fill_diagonal(M, rng.integers(4, 12, A))
    qs, ts = _weak_pairs(rng, [1100, 1300, 1500, 120, 300], ident=0.6, A=A, flank=(0, 40))
    b = _batch(qs, ts, M, 11, 1, "weak_protein_large", alphabet="ARNDCQEGHILKMFPSTWYV")
    compare(b, run_oracle(b), run_gpu_device(ctx, b))



def _one_gap_pairs(rng, npairs, A, gmax):
    """Query x+y against target x+z+y (and the roles swapped for every other
    pair), z a run of g letters, in random flanks: with z of a letter that
    matches nothing (A = 5) the optimum is the one-gap path, whose gap count is
    exactly the reverse band's bound G on its side and whose diagonals fill the
    traceback band [0, g] (or [-g, 0]) exactly.  Returns the pairs and each
    pair's (a, b, g)."""
    qs, ts, abg = [], [], []
    for p in range(npairs):
        g = int(rng.integers(1, gmax + 1))
        a, b = (int(v) for v in rng.integers(max(24, g + 4), 121, 2))
        x = rng.integers(0, 4, a).astype(np.uint8)
        y = rng.integers(0, 4, b).astype(np.uint8)
        z = (np.full(g, 4) if A == 5 else rng.integers(0, 4, g)).astype(np.uint8)
        gapped = np.concatenate([x, z, y])
        plain = np.concatenate([x, y])
        q, core = (plain, gapped) if p % 2 == 0 else (gapped, plain)
        ts.append(np.concatenate([rng.integers(0, 4, int(rng.integers(0, 50))), core,
                                  rng.integers(0, 4, int(rng.integers(0, 50)))]).astype(np.uint8))
        qs.append(q)
        abg.append((a, b, g))
    return qs, ts, np.array(abg)


@pytest.mark.parametrize("A,npairs", [(5, 17000), (4, 17000), (5, 3000)])
def test_one_gap_pairs_on_the_exact_band_edges(ctx, A, npairs):
    # 17,000 pairs take the thread-per-pair band kernel (reverse bands up to
    # 32 diagonals; wider ones the 16-bit reverse fill); 3,000 pairs the ring
    # reverse and the warp tracebacks; gaps of up to 40 letters cover every
    # traceback class of these lengths
    rng = np.random.default_rng(95 + A + npairs)
    qs, ts, abg = _one_gap_pairs(rng, npairs, A, 40)
    W = np.full((A, A), -3, np.int8)
    np.fill_diagonal(W, 2)
    b = _batch(qs, ts, W, 5, 2, f"one_gap_A{A}", alphabet="ACGTN"[:A])
    ora = run_oracle(b)
    if A == 5:
        # the construction holds: the one-gap optimum over the whole query
        res = ora[0]
        a, bb, g = abg.T
        assert (res["score1"] == 2 * (a + bb) - 5 - 2 * (g - 1)).all()
        assert (res["read_begin1"] == 0).all() and (res["read_end1"] == b.q_len - 1).all()
    compare(b, ora, run_gpu_device(ctx, b))


def test_banded_cta_reverse_on_the_band_edges(ctx):
    # long one-gap pairs (queries of 1,800-3,000 letters: the reversed fill
    # runs in the CTA kernel, each strip restricted to the reverse band's
    # columns): the one-gap optimum's gap count equals the band's bound on its
    # side, so the path touches the band's edge, and strips of 1,024 rows start
    # right of each other; plus exact self-alignments (a band of one diagonal)
    rng = np.random.default_rng(131)
    qs, ts = [], []
    for p, g in enumerate((1, 2, 17, 40, 200, 333, 1, 64)):
        a, b = (int(v) for v in rng.integers(900, 1501, 2))
        x = rng.integers(0, 4, a).astype(np.uint8)
        y = rng.integers(0, 4, b).astype(np.uint8)
        z = rng.integers(0, 4, g).astype(np.uint8)
        gapped, plain = np.concatenate([x, z, y]), np.concatenate([x, y])
        q, core = (plain, gapped) if p % 2 == 0 else (gapped, plain)
        qs.append(q)
        ts.append(np.concatenate([rng.integers(0, 4, int(rng.integers(0, 60))), core,
                                  rng.integers(0, 4, int(rng.integers(0, 60)))]).astype(np.uint8))
    for L in (1900, 2600):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q)
        ts.append(np.concatenate([rng.integers(0, 4, 40), q, rng.integers(0, 4, 25)]).astype(np.uint8))
    W = wl.dna_matrix(2, -3)
    b = _batch(qs, ts, W, 5, 2, "long_one_gap")
    assert (b.q_len > 1792).all()
    compare(b, run_oracle(b), run_gpu_device(ctx, b))


def test_host_io_colmax_at_callers_offsets(ctx):
    # host buffers: each pair's column maxima land at its own offset (here in
    # reverse pair order with gaps of 5 words), the words between the ranges
    # keep the caller's values, and a negative offset is refused
    b = mixed_dna(97, 300, 80, 400)
    ores, _, (ocm, ocmoff) = run_oracle(b)
    n = b.npairs
    cmoff = np.zeros(n, np.int64)
    at = 5
    for p in reversed(range(n)):
        cmoff[p] = at
        at += int(b.t_len[p]) + 5
    cm = np.full(at, -7, np.int32)
    res = np.zeros(n, gsw.RESULT_DTYPE)
    cap = int(b.q_len.sum() + b.t_len.sum() + 16)
    cig = np.zeros(cap, np.uint32)
    flags = gsw.GSW_CIGAR | gsw.GSW_COLMAX | gsw.GSW_HOST_IO
    rc = gsw.gsw_align_batch(ctx.handle, n, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                             b.gap_extend, flags, -1, res, cig, cap, cm, cmoff)
    assert rc == gsw.GSW_OK
    assert (res["score1"] == ores["score1"]).all() and (res["ref_end2"] == ores["ref_end2"]).all()
    inside = np.zeros(at, bool)
    for p in range(n):
        lo, L = int(cmoff[p]), int(b.t_len[p])
        assert np.array_equal(cm[lo:lo + L], ocm[ocmoff[p]:ocmoff[p] + L]), p
        inside[lo:lo + L] = True
    assert (cm[~inside] == -7).all()
    cmoff[3] = -1
    rc = gsw.gsw_align_batch(ctx.handle, n, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                             b.gap_extend, flags, -1, res, cig, cap, cm, cmoff, check=False)
    assert rc == gsw.GSW_EINVAL
