"""The allocation-free entry point (gsw_fill_static) against the oracle and the
regular entry point.

gsw_fill_static serves callers that must not allocate device memory; its
scratch is a fixed array inside the library.  These tests call it through the
C ABI twice in a row on the same device buffers and check every output
(scores, ends, secondary, per-column maxima) against the oracle on the same
inputs, and against gsw_align_batch.  All outputs are integers, so the
tolerance is zero.  Pairs the entry rejects (a target over its maximum, a
negative offset, a letter outside the alphabet) get the empty record flagged
GSW_RES_INVALID while the other pairs of the call are still aligned.  The file
is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1208_6350_gb300 import gsw, workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("score1", "score2", "ref_end1", "read_end1", "ref_end2")


def _pack(qs, ts, W, O, X, name, alphabet="ACGT"):
    ql = np.array([len(x) for x in qs], np.int32)
    tl = np.array([len(x) for x in ts], np.int32)
    qo = np.concatenate([[0], np.cumsum(ql)[:-1]]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(tl)[:-1]]).astype(np.int64)
    return wl.Batch(name, np.concatenate(qs).astype(np.uint8), qo, ql, np.concatenate(ts).astype(np.uint8), to,
                    tl, W, O, X, alphabet)


def _batch():
    b = wl.config2(3000, seed=21)
    b = b.subset(np.arange(b.npairs))
    rng = np.random.default_rng(4)
    # edge cases: empty query, empty target, length 1, and a target of
    # exactly the entry's maximum length
    q1024 = rng.integers(0, 4, 150).astype(np.uint8)
    t1024 = rng.integers(0, 4, gsw.GSW_STATIC_MAX_TARGET).astype(np.uint8)
    t1024[500:650] = q1024
    extra_q = [np.zeros(0, np.uint8), rng.integers(0, 4, 50).astype(np.uint8), np.array([2], np.uint8), q1024]
    extra_t = [rng.integers(0, 4, 80).astype(np.uint8), np.zeros(0, np.uint8), np.array([2], np.uint8), t1024]
    qs = [b.query(p) for p in range(b.npairs)] + extra_q
    ts = [b.target(p) for p in range(b.npairs)] + extra_t
    return _pack(qs, ts, b.W, 3, 1, "no_alloc")


def _oracle(b):
    res, _, (cm, _) = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                                         b.gap_extend, -1, colmax=True)
    assert (res["status"] == 0).all()
    return res, cm


def _dev(b, cmo=None):
    import torch
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    if cmo is None:
        cmo = np.zeros(b.npairs, np.int64)
        cmo[1:] = np.cumsum(b.t_len.astype(np.int64))[:-1]
    return dict(q=T(b.q), qo=T(b.q_off), ql=T(b.q_len), t=T(b.t), to=T(b.t_off), tl=T(b.t_len), cmo=T(cmo),
                total=max(int(b.t_len.clip(0).sum()), 1))


def _static(b, d, max_t=None, calls=2, expect=gsw.GSW_OK):
    import torch
    n = b.npairs
    outs = []
    for _ in range(calls):  # calls in a row share the static scratch
        res = torch.full((n * 12,), -7, dtype=torch.int32, device=d["q"].device)
        cm = torch.full((d["total"],), -7, dtype=torch.int32, device=d["q"].device)
        mt = int(b.t_len.max()) if max_t is None else max_t
        rc = gsw.gsw_fill_static(n, d["q"], d["qo"], d["ql"], d["t"], d["to"], d["tl"], mt, b.W, b.gap_open,
                                 b.gap_extend, gsw.GSW_COLMAX, -1, res, cm, d["cmo"])
        torch.cuda.synchronize()
        assert rc == expect, (gsw.strerror(rc), gsw.last_error())
        outs.append((res.cpu().numpy().view(gsw.RESULT_DTYPE), cm.cpu().numpy()))
    return outs


def _regular(b, d):
    import torch
    n = b.npairs
    ctx = gsw.Context(0, 2 << 30)
    try:
        ref = torch.zeros(n * 12, dtype=torch.int32, device=d["q"].device)
        ref_cm = torch.zeros(d["total"], dtype=torch.int32, device=d["q"].device)
        gsw.gsw_align_batch(ctx.handle, n, d["q"], d["qo"], d["ql"], d["t"], d["to"], d["tl"], b.W, b.gap_open,
                            b.gap_extend, gsw.GSW_COLMAX, -1, ref, None, 0, ref_cm, d["cmo"])
        torch.cuda.synchronize()
    finally:
        ctx.close()
    return ref.cpu().numpy().view(gsw.RESULT_DTYPE), ref_cm.cpu().numpy()


def _check_pairs(b, ores, ocm, res, cm, pairs, cmo=None):
    if cmo is None:
        cmo = np.zeros(b.npairs, np.int64)
        cmo[1:] = np.cumsum(b.t_len.astype(np.int64))[:-1]
    ocmo = np.zeros(b.npairs, np.int64)
    ocmo[1:] = np.cumsum(b.t_len.astype(np.int64))[:-1]
    for p in pairs:
        for f in FIELDS:
            assert int(res[f][p]) == int(ores[f][p]), (p, f, int(res[f][p]), int(ores[f][p]))
        assert res["ref_begin1"][p] == -1 and res["read_begin1"][p] == -1 and res["cigar_len"][p] == 0
        assert not (res["flags"][p] & (gsw.GSW_RES_INVALID | gsw.GSW_RES_INTERNAL))
        n = int(b.t_len[p])
        assert np.array_equal(cm[cmo[p]: cmo[p] + n], ocm[ocmo[p]: ocmo[p] + n]), p


def test_static_fill_matches_the_oracle_twice():
    b = _batch()
    ores, ocm = _oracle(b)
    d = _dev(b)
    outs = _static(b, d)
    for res, cm in outs:
        _check_pairs(b, ores, ocm, res, cm, range(b.npairs))
    # the same as the regular entry point, the 32-bit lane flag included
    ref, ref_cm = _regular(b, d)
    res, cm = outs[-1]
    for f in FIELDS:
        assert np.array_equal(res[f], ref[f]), f
    assert np.array_equal(res["flags"] & gsw.GSW_RES_S32, ref["flags"] & gsw.GSW_RES_S32)
    assert np.array_equal(cm, ref_cm)


def test_static_fill_32bit_refill_matches_the_oracle():
    rng = np.random.default_rng(8)
    qs, ts = [], []
    for L in (200, 326, 327, 400):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q)
        ts.append(np.concatenate([rng.integers(0, 4, 60), q, rng.integers(0, 4, 40)]).astype(np.uint8))
    b = _pack(qs, ts, wl.dna_matrix(100, -100), 30, 10, "ovf")
    ores, ocm = _oracle(b)
    outs = _static(b, _dev(b))
    for res, cm in outs:
        assert (res["flags"][2:] & gsw.GSW_RES_S32).all() and not (res["flags"][:2] & gsw.GSW_RES_S32).any()
        _check_pairs(b, ores, ocm, res, cm, range(b.npairs))


def test_static_fill_protein_queries_of_several_strips():
    # the general-alphabet kernel: 20 letters, a BLOSUM-range matrix, gap open
    # 11 / extend 1, queries past 256 rows (several strips of the 16-lane ring)
    ps = wl.protein_search(n_queries=40, n_db=60, seed=12)
    qidx = np.repeat(np.arange(40), 3)
    didx = np.random.default_rng(3).integers(0, 60, 120)
    b = ps.pairs(qidx, didx)
    keep = np.nonzero(b.t_len <= gsw.GSW_STATIC_MAX_TARGET)[0]
    b = b.subset(keep)
    assert (b.q_len > 256).sum() >= 10 and b.W.shape[0] == 20
    ores, ocm = _oracle(b)
    for res, cm in _static(b, _dev(b)):
        _check_pairs(b, ores, ocm, res, cm, range(b.npairs))


def test_static_fill_rejects_bad_pairs_and_aligns_the_rest():
    b = _batch()
    ores, ocm = _oracle(b)
    rng = np.random.default_rng(9)
    # pair 7: a target of max + 1 letters (allowed by max_target_len, caught by
    # the kernel); pair 11: a negative target offset; pair 13: a letter code 4;
    # pair 17: a negative max-array offset
    long_t = rng.integers(0, 4, gsw.GSW_STATIC_MAX_TARGET + 1).astype(np.uint8)
    t = np.concatenate([b.t, long_t])
    t_off = b.t_off.copy()
    t_len = b.t_len.copy()
    t_off[7], t_len[7] = len(b.t), len(long_t)
    t_off[11] = -5
    q = b.q.copy()
    q[b.q_off[13]] = 4
    bad = wl.Batch("bad", q, b.q_off, b.q_len, t, t_off, t_len, b.W, 3, 1, "ACGT")
    cmo = np.zeros(b.npairs, np.int64)
    cmo[1:] = np.cumsum(t_len.astype(np.int64))[:-1]
    cmo[17] = -1
    d = _dev(bad, cmo)
    d["total"] = int(cmo.max() + t_len.max() + 1)
    outs = _static(bad, d, max_t=gsw.GSW_STATIC_MAX_TARGET, expect=gsw.GSW_EINVAL)
    assert "GSW_RES_INVALID" in gsw.last_error()
    rejected = [7, 11, 13, 17]
    for res, cm in outs:
        for p in rejected:
            assert res["flags"][p] & gsw.GSW_RES_INVALID, p
            assert res["score1"][p] == 0 and res["ref_end1"][p] == -1 and res["read_end1"][p] == -1
        good = [p for p in range(b.npairs) if p not in rejected]
        _check_pairs(b, ores, ocm, res, cm, good, cmo)
