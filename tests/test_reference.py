"""Reads against one long reference (gsw_align_to_reference): every record and
CIGAR equals the oracle's for the pair (read, whole reference), with windows
small enough that alignments, masks and overlaps straddle window boundaries."""
import numpy as np
import pytest

import oracle
from paper_1208_6350_gb300 import gsw, workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")


def _reads_and_reference(seed, n_ref=50000, window=2048):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 4, n_ref).astype(np.uint8)
    reads = []

    def mutate(s):
        s = s.copy()
        mut = rng.random(len(s)) < 0.03
        s[mut] = rng.integers(0, 4, int(mut.sum()))
        return s

    for k in range(36):
        L = int(rng.integers(60, 250))
        kind = k % 6
        if kind == 0:      # random read: no real alignment
            r = rng.integers(0, 4, L).astype(np.uint8)
        elif kind == 1:    # copy straddling a window boundary
            b = int(rng.integers(1, n_ref // window)) * window
            o = max(0, min(n_ref - L, b - L // 2))
            r = mutate(ref[o:o + L])
        elif kind == 2:    # near the reference start or end
            o = 0 if k % 4 == 2 else n_ref - L
            r = mutate(ref[o:o + L])
        elif kind == 3:    # two exact copies far apart: score2 == score1 outside the mask
            o = int(rng.integers(0, n_ref - L))
            r = ref[o:o + L].copy()
            o2 = (o + n_ref // 2) % (n_ref - L)
            ref[o2:o2 + L] = r
        elif kind == 4:    # a second copy just past the mask, possibly in the next window
            o = int(rng.integers(0, n_ref - 3 * L))
            r = ref[o:o + L].copy()
            o2 = o + L + L // 2 + 20
            ref[o2:o2 + L] = mutate(r)
        else:              # an ordinary placed read
            o = int(rng.integers(0, n_ref - L))
            r = mutate(ref[o:o + L])
        reads.append(r)
    q_len = np.array([len(r) for r in reads], np.int32)
    q_off = np.concatenate([[0], np.cumsum(q_len)[:-1]]).astype(np.int64)
    return np.concatenate(reads), q_off, q_len, ref


@pytest.mark.parametrize("window", [2048, 5000, 0])
def test_reads_against_reference_equal_whole_reference_oracle(window):
    q, q_off, q_len, ref = _reads_and_reference(71)
    W = wl.dna_matrix(2, -3)
    O, X = 5, 2
    ctx = gsw.Context(0, 4 << 30)
    try:
        res, cig, rc = ctx.align_to_reference(q, q_off, q_len, ref, W, O, X, gsw.GSW_CIGAR, -1, window)
    finally:
        ctx.close()
    assert rc == gsw.GSW_OK
    n = len(q_len)
    t_off = np.zeros(n, np.int64)
    t_len = np.full(n, len(ref), np.int32)
    ores, ocg, _ = oracle.align_batch(q, q_off, q_len, ref, t_off, t_len, W, O, X,
                                      cigar_stride=int(q_len.max() + len(ref) + 2))
    for p in range(n):
        for f in FIELDS:
            assert int(res[f][p]) == int(ores[f][p]), (window, p, f, int(res[f][p]), int(ores[f][p]))
        assert not (res["flags"][p] & 0x80)
        want = oracle.decode_cigar(ocg[p, : ores["cigar_len"][p]])
        got = oracle.decode_cigar(cig[res["cigar_off"][p]: res["cigar_off"][p] + res["cigar_len"][p]]) \
            if res["cigar_len"][p] > 0 else []
        assert got == want, (window, p)
    # the constructions did what they claim
    assert (ores["score2"] == ores["score1"]).any()


def test_window_smaller_than_mask_and_overlap_rejected():
    q, q_off, q_len, ref = _reads_and_reference(72, n_ref=8000)
    ctx = gsw.Context(0, 1 << 30)
    try:
        _, _, rc = ctx.align_to_reference(q, q_off, q_len, ref, wl.dna_matrix(2, -3), 5, 2, gsw.GSW_CIGAR, -1, 64)
    finally:
        ctx.close()
    assert rc == gsw.GSW_EINVAL


def test_device_inputs_written_on_the_callers_stream():
    # device arrays and a non-default stream: the read lengths are written by
    # work queued on that stream just before the call (behind a ~20 ms delay
    # kernel), so the call must read them on the same stream
    import torch
    q, q_off, q_len, ref = _reads_and_reference(73)
    W = wl.dna_matrix(2, -3)
    O, X = 5, 2
    n = len(q_len)
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dq, dqo, dref, ql_src = T(q), T(q_off), T(ref), T(q_len)
    dql = torch.zeros(n, dtype=torch.int32, device=dev)
    cap = int(2 * q_len.sum() + 64 * n + 64)
    dres = torch.zeros(n * gsw.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    dcig = torch.zeros(cap, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    ctx = gsw.Context(0, 4 << 30)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            torch.cuda._sleep(40_000_000)
            dql.copy_(ql_src)
            rc = gsw.load().gsw_align_to_reference(
                ctx.handle, n, dq.data_ptr(), dqo.data_ptr(), dql.data_ptr(), dref.data_ptr(), len(ref),
                W.ctypes.data, 4, O, X, gsw.GSW_CIGAR, -1, 2048, dres.data_ptr(), dcig.data_ptr(), cap,
                s.cuda_stream)
        s.synchronize()
    finally:
        ctx.close()
    assert rc == gsw.GSW_OK
    res = dres.cpu().numpy().view(gsw.RESULT_DTYPE)
    cig = dcig.cpu().numpy().view(np.uint32)
    t_off = np.zeros(n, np.int64)
    t_len = np.full(n, len(ref), np.int32)
    ores, ocg, _ = oracle.align_batch(q, q_off, q_len, ref, t_off, t_len, W, O, X,
                                      cigar_stride=int(q_len.max() + len(ref) + 2))
    for p in range(n):
        for f in FIELDS:
            assert int(res[f][p]) == int(ores[f][p]), (p, f, int(res[f][p]), int(ores[f][p]))
        want = oracle.decode_cigar(ocg[p, : ores["cigar_len"][p]])
        got = oracle.decode_cigar(cig[res["cigar_off"][p]: res["cigar_off"][p] + res["cigar_len"][p]]) \
            if res["cigar_len"][p] > 0 else []
        assert got == want, p
