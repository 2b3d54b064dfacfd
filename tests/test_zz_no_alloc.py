"""The allocation-free entry point (gsw_fill_static) against the regular one.

gsw_fill_static serves callers that must not allocate device memory; its
scratch is a fixed array inside the library.  This test calls it through the
C ABI twice in a row on the same device buffers and checks every output
(scores, ends, secondary, per-column maxima) against gsw_align_batch on the
same inputs.  All outputs are integers, so the tolerance is zero.  The file is
named to be collected last.
"""
import numpy as np
import pytest

from paper_1208_6350_gb300 import gsw, workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("score1", "score2", "ref_end1", "read_end1", "ref_end2", "ref_begin1", "read_begin1",
          "cigar_len")


def _batch():
    b = wl.config2(3000, seed=21)
    b = b.subset(np.arange(b.npairs))
    rng = np.random.default_rng(4)
    # edge cases: empty query, empty target, length 1, and pairs whose score
    # overflows 16-bit lanes under a large match score
    extra_q = [np.zeros(0, np.uint8), rng.integers(0, 4, 50).astype(np.uint8), np.array([2], np.uint8)]
    extra_t = [rng.integers(0, 4, 80).astype(np.uint8), np.zeros(0, np.uint8), np.array([2], np.uint8)]
    qs = [b.query(p) for p in range(b.npairs)] + extra_q
    ts = [b.target(p) for p in range(b.npairs)] + extra_t
    ql = np.array([len(x) for x in qs], np.int32)
    tl = np.array([len(x) for x in ts], np.int32)
    qo = np.concatenate([[0], np.cumsum(ql)[:-1]]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(tl)[:-1]]).astype(np.int64)
    return wl.Batch("no_alloc", np.concatenate(qs), qo, ql, np.concatenate(ts), to, tl, b.W, 3, 1, "ACGT")


def _run_both(b, W, O, X):
    import torch
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    q, t, qo, to = T(b.q), T(b.t), T(b.q_off), T(b.t_off)
    ql, tl = T(b.q_len), T(b.t_len)
    n = b.npairs
    cmo = np.zeros(n, np.int64)
    cmo[1:] = np.cumsum(b.t_len.astype(np.int64))[:-1]
    cmo_d = T(cmo)
    total = max(int(b.t_len.sum()), 1)
    ctx = gsw.Context(0, 2 << 30)
    try:
        ref = torch.zeros(n * 12, dtype=torch.int32, device=dev)
        ref_cm = torch.zeros(total, dtype=torch.int32, device=dev)
        gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, W, O, X, gsw.GSW_COLMAX, -1, ref, None, 0,
                            ref_cm, cmo_d)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        res = torch.full((n * 12,), -7, dtype=torch.int32, device=dev)
        cm = torch.full((total,), -7, dtype=torch.int32, device=dev)
        rc = gsw.gsw_fill_static(n, q, qo, ql, t, to, tl, int(b.t_len.max()), W, O, X, gsw.GSW_COLMAX,
                                 -1, res, cm, cmo_d)
        torch.cuda.synchronize()
        assert rc == gsw.GSW_OK, gsw.strerror(rc)
        outs.append((res.cpu().numpy().view(gsw.RESULT_DTYPE), cm.cpu().numpy()))
    return ref.cpu().numpy().view(gsw.RESULT_DTYPE), ref_cm.cpu().numpy(), outs


def test_static_fill_matches_regular_entry_twice():
    b = _batch()
    ref, ref_cm, outs = _run_both(b, b.W, 3, 1)
    for res, cm in outs:
        for f in FIELDS:
            assert np.array_equal(res[f], ref[f]), f
        assert np.array_equal(res["flags"] & gsw.GSW_RES_S32, ref["flags"] & gsw.GSW_RES_S32)
        assert np.array_equal(cm, ref_cm)


def test_static_fill_32bit_refill_matches():
    rng = np.random.default_rng(8)
    qs, ts = [], []
    for L in (200, 326, 327, 400):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q)
        ts.append(np.concatenate([rng.integers(0, 4, 60), q, rng.integers(0, 4, 40)]).astype(np.uint8))
    ql = np.array([len(x) for x in qs], np.int32)
    tl = np.array([len(x) for x in ts], np.int32)
    b = wl.Batch("ovf", np.concatenate(qs), np.concatenate([[0], np.cumsum(ql)[:-1]]).astype(np.int64), ql,
                 np.concatenate(ts), np.concatenate([[0], np.cumsum(tl)[:-1]]).astype(np.int64), tl,
                 wl.dna_matrix(100, -100), 30, 10, "ACGT")
    ref, ref_cm, outs = _run_both(b, b.W, 30, 10)
    assert (ref["flags"][2:] & gsw.GSW_RES_S32).all()
    for res, cm in outs:
        for f in FIELDS:
            assert np.array_equal(res[f], ref[f]), f
        assert np.array_equal(cm, ref_cm)


def test_static_fill_rejects_targets_beyond_its_maximum():
    W = wl.dna_matrix(2, -2)
    rc = gsw.gsw_fill_static(1, 1, 1, 1, 1, 1, 1, gsw.GSW_STATIC_MAX_TARGET + 1, W, 3, 1)
    assert rc == gsw.GSW_EINVAL
