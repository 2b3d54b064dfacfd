"""Serving loop: each request's results are the same alone and in the mix.

Requests of mixed sizes (short reads, short-read extensions, scaled-down long
reads) are submitted from two threads at once; every request's records and
CIGAR must equal (zero tolerance) what gsw_align_batch gives for that request
alone, and the oracle's.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_1208_6350_gb300 import gsw, workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        kind = rng.choice(3, p=[0.6, 0.3, 0.1])
        npairs = int(rng.integers(1, 17))
        s = int(rng.integers(0, 2**31 - 1))
        if kind == 0:
            b = wl.dna_short_reads(npairs, (100, 100), (1000, 1000), 0.02, 0.002, 3, seed=s)
        elif kind == 1:
            b = wl.dna_short_reads(npairs, (100, 250), (300, 1000), 0.01, 0.001, 3, 0.10, seed=s)
        else:
            b = wl.dna_long_reads(min(npairs, 3), 400, 1500, seed=s)
            b = wl.Batch(b.name, b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, wl.dna_matrix(2, -2), 3, 1, "ACGT")
        reqs.append(b)
    return reqs


def _decode(res, cig, p):
    n, o = int(res["cigar_len"][p]), int(res["cigar_off"][p])
    return oracle.decode_cigar(cig[o:o + n]) if n > 0 else []


@pytest.mark.parametrize("heavy_cells", [0, 1 << 20])
def test_mixed_stream_equals_alone_and_oracle(heavy_cells):
    # heavy_cells 2^20: the long-read requests queue apart for the heavy
    # workers (launches capped at 7/8 of the SMs)
    reqs = _requests(60, 3)
    W = wl.dna_matrix(2, -2)
    srv = gsw.Server(W, 3, 1, gsw.GSW_CIGAR, workers=3, max_batch_pairs=256, max_batch_letters=1 << 20,
                     mem_budget_bytes=3 << 30, heavy_cells=heavy_cells)
    ids = [None] * len(reqs)

    def submit(lo, hi):
        for k in range(lo, hi):
            b = reqs[k]
            ids[k] = srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len)

    th = [threading.Thread(target=submit, args=(0, 30)), threading.Thread(target=submit, args=(30, 60))]
    for x in th:
        x.start()
    for x in th:
        x.join()
    got = []
    for k, b in enumerate(reqs):
        rc, res, cig, tm = srv.poll(ids[k], b.npairs, times=True)
        assert rc == gsw.GSW_OK
        assert 0 <= tm[0] <= tm[1] <= tm[2] <= srv.now()
        got.append((res, cig))
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["batches"] >= 2

    ctx = gsw.Context(0, 2 << 30)
    try:
        for k, b in enumerate(reqs):
            alone, acig, _, rc = ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, W, 3, 1,
                                                gsw.GSW_CIGAR, -1, int(b.q_len.sum() + b.t_len.sum() + 64))
            ores, ocg, _ = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, W, 3, 1,
                                              cigar_stride=int(b.q_len.max() + b.t_len.max() + 2))
            res, cig = got[k]
            for p in range(b.npairs):
                for f in FIELDS:
                    assert int(res[f][p]) == int(alone[f][p]) == int(ores[f][p]), (k, p, f)
                want = oracle.decode_cigar(ocg[p, : ores["cigar_len"][p]])
                assert _decode(res, cig, p) == _decode(alone, acig, p) == want, (k, p)
    finally:
        ctx.close()


def test_poll_timeout_unknown_id_and_bad_letters():
    W = wl.dna_matrix(2, -2)
    srv = gsw.Server(W, 3, 1, gsw.GSW_CIGAR, workers=2, max_batch_pairs=64, max_batch_letters=1 << 20,
                     mem_budget_bytes=2 << 30)
    try:
        reqs = _requests(12, 5)
        ids = [srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len) for b in reqs]
        rc, res, _ = srv.poll(ids[-1], reqs[-1].npairs, timeout_us=0)
        assert rc == gsw.GSW_ETIMEDOUT and res is None
        for k, b in enumerate(reqs):
            rc, res, _ = srv.poll(ids[k], b.npairs, timeout_us=20_000_000)
            assert rc == gsw.GSW_OK
        rc, _, _ = srv.poll(123456789, 1, timeout_us=0)
        assert rc == gsw.GSW_ENOTFOUND
        b = reqs[0]
        bad = b.t.copy()
        bad[0] = 9
        with pytest.raises(gsw.GswError) as ei:
            srv.submit(b.q, b.q_off, b.q_len, bad, b.t_off, b.t_len)
        assert ei.value.code == gsw.GSW_EINVAL
    finally:
        srv.close()


@pytest.mark.parametrize("light_graphs", [0, -1])
def test_light_batches_replay_captured_graphs(light_graphs):
    # one worker, requests of similar shape served one after the other: with
    # graphs on, batches padded to 64 pairs and bucketed lengths repeat one
    # captured pipeline (replayed from the third batch on); with graphs off
    # every batch launches eagerly.  Records and CIGARs equal the oracle's
    # either way.
    W = wl.dna_matrix(2, -2)
    srv = gsw.Server(W, 3, 1, gsw.GSW_CIGAR, workers=1, max_batch_pairs=256, max_batch_letters=1 << 20,
                     mem_budget_bytes=2 << 30, heavy_workers=-1, light_graphs=light_graphs)
    try:
        reqs = [wl.dna_short_reads(int(n), (200, 250), (900, 1000), 0.01, 0.001, 3, 0.10, seed=40 + k)
                for k, n in enumerate([5, 9, 17, 3, 30, 12, 8, 21, 2, 16])]
        got = []
        for b in reqs:
            rid = srv.submit(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len)
            rc, res, cig = srv.poll(rid, b.npairs, timeout_us=30_000_000)
            assert rc == gsw.GSW_OK
            got.append((res, cig))
        st = srv.stats()
    finally:
        srv.close()
    assert st["batches"] == len(reqs)
    if light_graphs >= 0:
        assert st["graph_batches"] >= 3
    else:
        assert st["graph_batches"] == 0
    for b, (res, cig) in zip(reqs, got):
        ores, ocg, _ = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, W, 3, 1,
                                          cigar_stride=int(b.q_len.max() + b.t_len.max() + 2))
        for p in range(b.npairs):
            for f in FIELDS:
                assert int(res[f][p]) == int(ores[f][p]), (p, f)
            assert _decode(res, cig, p) == oracle.decode_cigar(ocg[p, : ores["cigar_len"][p]])
