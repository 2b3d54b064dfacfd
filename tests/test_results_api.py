"""GPU checks of the library-owned results (gsw_align_batch_results,
gsw_results_get / gsw_results_free, gsw_serve_poll_results): the handle's
records, CIGARs and max arrays equal the oracle's for host and device inputs,
including a batch whose CIGAR words outgrow the first buffer the library
reserves, and a served request returned as a handle."""
import numpy as np
import pytest

import oracle
from paper_1208_6350_gb300 import gsw, workloads as wl
from parity_util import FIELDS, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gsw.Context(0, 4 << 30)
    yield c
    c.close()


def _check_handle(b, ora, h, colmax=True):
    ores, ocg, ocm = ora
    assert gsw.gsw_results_count(h) == b.npairs
    for p in range(b.npairs):
        r = gsw.gsw_results_get(h, p)
        for f in FIELDS:
            assert r[f] == int(ores[f][p]), (p, f)
        assert r["lane_bits_used"] in (16, 32) and r["n"] == int(b.t_len[p])
        assert r["cigar"] == [(int(w) >> 4, int(w) & 15) for w in ocg[p, : ores["cigar_len"][p]]], p
        if colmax:
            cm, cmoff = ocm
            want = cm[cmoff[p]: cmoff[p] + b.t_len[p]]
            got = r["colmax"] if r["colmax"] is not None else np.zeros(0, np.int32)
            assert np.array_equal(got, want), p


def _dev_args(b):
    import torch
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return T(b.q), T(b.q_off), T(b.q_len), T(b.t), T(b.t_off), T(b.t_len)


def test_results_handle_host_inputs(ctx):
    b = wl.config1().subset(np.arange(200))
    ora = run_oracle(b)
    rc, h = gsw.gsw_align_batch_results(ctx.handle, b.npairs, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W,
                                        b.gap_open, b.gap_extend,
                                        gsw.GSW_CIGAR | gsw.GSW_COLMAX | gsw.GSW_HOST_IO)
    assert rc == gsw.GSW_OK and h
    try:
        _check_handle(b, ora, h)
    finally:
        gsw.gsw_results_free(h)


def test_results_handle_device_inputs_and_cigar_regrowth(ctx):
    # reads at 16 % indels: hundreds of CIGAR runs per pair, more than the
    # words the library reserves first (a sixteenth of the shorter sequence
    # per pair), so the pairs that did not fit are aligned again on their
    # own; mixed with short pairs that fit at once
    lb = wl.dna_long_reads(8, 2000, 4000, p_sub=0.04, p_ins=0.08, p_del=0.08, seed=41)
    sb = wl.config2(40, seed=42)
    b = wl.concat([lb, sb.subset(np.arange(sb.npairs))])
    b = wl.Batch(b.name, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, lb.W, lb.gap_open, lb.gap_extend, "ACGT")
    ora = run_oracle(b)
    first = 1024 + int((np.minimum(b.q_len, b.t_len) // 16 + 4).sum())
    assert int(ora[0]["cigar_len"].sum()) > first  # the first reservation overflows
    rc, h = gsw.gsw_align_batch_results(ctx.handle, b.npairs, *_dev_args(b), b.W, b.gap_open, b.gap_extend,
                                        gsw.GSW_CIGAR | gsw.GSW_COLMAX)
    assert rc == gsw.GSW_OK and h
    try:
        _check_handle(b, ora, h)
    finally:
        gsw.gsw_results_free(h)
    # the same with host inputs
    rc, h = gsw.gsw_align_batch_results(ctx.handle, b.npairs, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W,
                                        b.gap_open, b.gap_extend, gsw.GSW_CIGAR | gsw.GSW_HOST_IO)
    assert rc == gsw.GSW_OK and h
    try:
        _check_handle(b, ora, h, colmax=False)
    finally:
        gsw.gsw_results_free(h)


def test_results_handle_score_only(ctx):
    b = wl.config2(500, seed=43)
    b = b.subset(np.arange(b.npairs))
    ores, _, _ = run_oracle(b)
    rc, h = gsw.gsw_align_batch_results(ctx.handle, b.npairs, *_dev_args(b), b.W, b.gap_open, b.gap_extend, 0)
    assert rc == gsw.GSW_OK
    try:
        for p in range(b.npairs):
            r = gsw.gsw_results_get(h, p)
            for f in ("score1", "score2", "ref_end1", "read_end1", "ref_end2"):
                assert r[f] == int(ores[f][p])
            assert r["cigar"] == [] and r["colmax"] is None and r["ref_begin1"] == -1
        with pytest.raises(gsw.GswError):
            gsw.gsw_results_get(h, b.npairs)
    finally:
        gsw.gsw_results_free(h)


def test_served_request_as_a_handle():
    b = wl.config1().subset(np.arange(40))
    ora = run_oracle(b)
    srv = gsw.Server(b.W, b.gap_open, b.gap_extend, flags=gsw.GSW_CIGAR, workers=2)
    try:
        rid = srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len)
        rc, h = srv.poll_results(rid, 30_000_000)
        assert rc == gsw.GSW_OK and h
        try:
            _check_handle(b, ora, h, colmax=False)
        finally:
            gsw.gsw_results_free(h)
        rc, h = srv.poll_results(rid, 0)  # forgotten once returned
        assert rc == gsw.GSW_ENOTFOUND and not h
    finally:
        srv.close()
