"""CPU checks of bench.py's host-side summary of the work beside the forward
fill (32-bit refills, reversed rectangle, begin-end region): hand-made records
with known counts, and invariants on the oracle's records of a sample of the
short-read extension workload."""
import numpy as np

import bench
import oracle
from paper_1208_6350_gb300 import gsw


def _records(rows):
    r = np.zeros(len(rows), gsw.RESULT_DTYPE)
    for k, (s1, rb, re, tb, te, fl) in enumerate(rows):
        r[k]["score1"], r[k]["read_begin1"], r[k]["read_end1"] = s1, rb, re
        r[k]["ref_begin1"], r[k]["ref_end1"], r[k]["flags"] = tb, te, fl
    return r


def test_counts_on_hand_made_records():
    r = _records([(10, 2, 5, 3, 9, 0x1),       # rect 6 x 7, region 4 x 7, 32-bit
                  (0, -1, -1, -1, -1, 0),      # no alignment: counted nowhere
                  (5, 0, 0, 0, 0, 0x2)])       # 1 x 1; CIGAR-space flag is not 32-bit
    w = bench.work_summary(r, 100)
    assert w["pairs"] == 3 and w["aligned_pairs"] == 2
    assert w["s32_refill_pairs"] == 1 and w["s32_refill_frac"] == round(1 / 3, 4)
    assert w["reverse_rect_cells"] == 42 + 1 and w["reverse_rect_frac"] == 0.43
    assert w["region_cells"] == 28 + 1 and w["region_frac"] == 0.29


def test_invariants_on_oracle_records():
    b, _ = bench.make_workload("dna_short_read_extension_1M", 2000, 0)
    ores, _, _ = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                                    b.gap_extend)
    r = np.zeros(b.npairs, gsw.RESULT_DTYPE)
    for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2"):
        r[f] = ores[f]
    w = bench.work_summary(r, b.cells)
    # the region lies inside the reversed rectangle, which lies inside the pair
    assert 0 < w["region_cells"] <= w["reverse_rect_cells"] <= b.cells
    # decoys (10 %) still align somewhere; true reads align over most of the read
    assert w["aligned_pairs"] == int((ores["score1"] > 0).sum())
    assert 0.05 < w["region_frac"] < 0.5


class _OracleContext:
    """Stands in for gsw.Context.align_host: the oracle's records in the
    library's record layout (no GPU)."""

    def __init__(self):
        self.calls = []

    def align_host(self, q, q_off, q_len, t, t_off, t_len, W, O, X, flags, mask_len, cap):
        self.calls.append((len(q_len), flags))
        o, _, _ = oracle.align_batch(q, q_off, q_len, t, t_off, t_len, W, O, X, mask_len)
        r = np.zeros(len(q_len), gsw.RESULT_DTYPE)
        for f in ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2"):
            r[f] = o[f]
        return r, np.zeros(max(cap, 1), np.uint32), (None, None), gsw.GSW_OK


def test_plain_per_pair_leg_reports_and_compares():
    b, _ = bench.make_workload("dna_short_read_extension_1M", 300, 0)
    ctx = _OracleContext()
    batched = ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open, b.gap_extend,
                             gsw.GSW_CIGAR, -1, 0)[0]
    out = bench.run_plain(gsw, b, ctx, 120, batched)
    assert out["pairs"] == 120 and out["same_records_as_batched"] is True
    assert out["cells"] == int((b.q_len[:120].astype(np.int64) * b.t_len[:120]).sum())
    # a warm-up call, then one call over the pairs, both on the plain path
    assert [c[0] for c in ctx.calls[1:]] == [8, 120]
    assert all(c[1] & gsw.GSW_PLAIN for c in ctx.calls[1:])
    batched = batched.copy()
    batched["score1"][5] += 1
    assert bench.run_plain(gsw, b, ctx, 120, batched)["same_records_as_batched"] is False
