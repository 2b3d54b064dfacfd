"""GPU parity on long reads at the full lengths of the long-read workload.

The long-read workload (10 % error: 6 % substitutions, 2 % insertions, 2 %
deletions; +2/-4, gap open 4, extend 2; targets 1.2x the read) runs reads of
up to 20 kb.  Here four reads of 15-20 kb take every stage at that size:
forward fills of 30-40 strips of 512 rows in the CTA kernel, the reversed
fill, and the wide-band traceback (bands of thousands of diagonals, the strip
kernel).  A second run on a context with a small memory budget makes the
traceback's direction-word pool smaller than the batch's words, so its pairs
run in at least two groups that reuse the pool one after the other (checked
through gsw_last_stats).  Every field, the CIGAR and the max array are
compared with the oracle's, with zero tolerance.
"""
import numpy as np
import pytest

from paper_1208_6350_gb300 import gsw, workloads as wl
from parity_util import compare, run_gpu_device, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch_and_oracle():
    b = wl.dna_long_reads(4, 15000, 20000, seed=31)
    assert b.q_len.min() >= 14000 and b.q_len.max() <= 21000
    return b, run_oracle(b)


def test_full_length_long_reads_every_output(batch_and_oracle):
    b, ora = batch_and_oracle
    ctx = gsw.Context(0, 8 << 30)
    try:
        got = run_gpu_device(ctx, b)
        st = gsw.gsw_last_stats(ctx.handle)
    finally:
        ctx.close()
    compare(b, ora, got)
    # reads of 30-40 strips of 512 rows; their bands exceed 512 diagonals
    assert (b.q_len > 30 * 512 - 1).sum() >= 2
    assert st["ring_words"] > 0 and st["internal_pairs"] == 0


def test_wide_band_traceback_in_several_pool_groups(batch_and_oracle):
    b, ora = batch_and_oracle
    # shrink the context's budget until the traceback pool cannot hold every
    # pair's direction words at once (ring_words > ring_pool_words: two or
    # more groups), then compare everything once more
    budget = 4 << 30
    hit = None
    while budget > (64 << 20):
        ctx = gsw.Context(0, budget)
        try:
            try:
                got = run_gpu_device(ctx, b)
            except gsw.GswError as e:
                if e.code != gsw.GSW_ENOMEM:
                    raise
                break  # the budget no longer holds one pair's words
            st = gsw.gsw_last_stats(ctx.handle)
        finally:
            ctx.close()
        if st["ring_words"] > st["ring_pool_words"] > 0:
            hit = (got, st, budget)
            break
        budget = int(budget * 0.8)
    assert hit is not None, "no budget split the wide-band traceback into groups"
    got, st, budget = hit
    assert st["ring_groups"] >= 2
    compare(b, ora, got)
