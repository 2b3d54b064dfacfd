"""All-vs-all (gsw_align_all_pairs): record k of the row-major triangle equals
the oracle's record for the pair (i, j), i < j, with chunks smaller than the
triangle (pair generation across chunk boundaries, CIGAR offsets of later
chunks) and 2-bit packed input."""
import numpy as np
import pytest

import oracle
from paper_1208_6350_gb300 import gsw, workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")


def _reads(seed, n=70):
    # overlapping fragments of one random genome, 50-90 nt, some reversed
    # order of appearance: many true overlaps and many unrelated pairs
    rng = np.random.default_rng(seed)
    genome = rng.integers(0, 4, 3000).astype(np.uint8)
    reads = []
    for _ in range(n):
        L = int(rng.integers(50, 90))
        o = int(rng.integers(0, len(genome) - L))
        r = genome[o:o + L].copy()
        mut = rng.random(L) < 0.02
        r[mut] = rng.integers(0, 4, int(mut.sum()))
        reads.append(r)
    ln = np.array([len(r) for r in reads], np.int32)
    off = np.concatenate([[0], np.cumsum(ln)[:-1]]).astype(np.int64)
    return np.concatenate(reads), off, ln


@pytest.mark.parametrize("chunk,packed", [(0, False), (777, False), (1000, True)])
def test_all_pairs_equal_oracle(chunk, packed):
    seq, off, ln = _reads(81)
    n = len(ln)
    W = wl.dna_matrix(2, -3)
    ctx = gsw.Context(0, 2 << 30)
    try:
        s = gsw.pack2(seq) if packed else seq
        flags = gsw.GSW_CIGAR | (gsw.GSW_PACKED2 if packed else 0)
        res, cig, rc = ctx.align_all_pairs(s, off, ln, W, 5, 2, flags, -1, chunk)
    finally:
        ctx.close()
    assert rc == gsw.GSW_OK
    ii, jj = np.triu_indices(n, 1)
    assert len(res) == len(ii)
    ores, ocg, _ = oracle.align_batch(seq, off[ii], ln[ii], seq, off[jj], ln[jj], W, 5, 2,
                                      cigar_stride=int(2 * ln.max() + 2))
    for f in FIELDS:
        bad = np.nonzero(res[f] != ores[f])[0]
        assert len(bad) == 0, (f, bad[:5])
    for k in range(len(ii)):
        want = oracle.decode_cigar(ocg[k, : ores["cigar_len"][k]])
        o, c = int(res["cigar_off"][k]), int(res["cigar_len"][k])
        got = oracle.decode_cigar(cig[o:o + c]) if c > 0 else []
        assert got == want, k
    assert (ores["score1"] > 60).sum() > 20  # real overlaps among the pairs


def test_all_pairs_score_only():
    seq, off, ln = _reads(82, n=40)
    W = wl.dna_matrix(2, -3)
    ctx = gsw.Context(0, 1 << 30)
    try:
        res, _, rc = ctx.align_all_pairs(seq, off, ln, W, 5, 2, 0)
    finally:
        ctx.close()
    assert rc == gsw.GSW_OK
    ii, jj = np.triu_indices(len(ln), 1)
    ores, _, _ = oracle.align_batch(seq, off[ii], ln[ii], seq, off[jj], ln[jj], W, 5, 2,
                                    cigar_stride=int(2 * ln.max() + 2))
    for f in ("score1", "score2", "ref_end1", "read_end1", "ref_end2"):
        assert (res[f] == ores[f]).all(), f
    assert (res["cigar_len"] == 0).all() and (res["ref_begin1"] == -1).all()
