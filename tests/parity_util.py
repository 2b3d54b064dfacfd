"""Helpers for the GPU parity tests: run both sides on the same seeded batch
and compare every output element by element (all outputs are integers, so
the tolerance is zero)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1208_6350_gb300 import gsw

FIELDS = ("score1", "score2", "ref_begin1", "ref_end1", "read_begin1", "read_end1", "ref_end2")


def run_oracle(b, mask_len=-1, colmax=True):
    stride = int((b.q_len.max(initial=0) + b.t_len.max(initial=0)) + 2)
    res, cg, cm = oracle.align_batch(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W, b.gap_open,
                                     b.gap_extend, mask_len, cigar_stride=stride, colmax=colmax)
    assert (res["status"] == 0).all(), "oracle reported a failure"
    return res, cg, cm


def run_gpu_host(ctx, b, flags=gsw.GSW_CIGAR, mask_len=-1, colmax=True):
    cap = int(b.q_len.sum() + b.t_len.sum() + 16)
    res, cig, (cm, cmoff), rc = ctx.align_host(b.q, b.q_off, b.q_len, b.t, b.t_off, b.t_len, b.W,
                                               b.gap_open, b.gap_extend, flags, mask_len, cap, colmax)
    assert rc == gsw.GSW_OK, rc
    return res, cig, (cm, cmoff)


def run_gpu_device(ctx, b, flags=gsw.GSW_CIGAR, mask_len=-1, colmax=True, stream=None):
    """Device-resident inputs and outputs (torch tensors), the bench's path."""
    import torch
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n = b.npairs
    q, t = T(b.q), T(b.t)
    qo, to = T(b.q_off.astype(np.int64)), T(b.t_off.astype(np.int64))
    ql, tl = T(b.q_len.astype(np.int32)), T(b.t_len.astype(np.int32))
    res = torch.zeros(n * 12, dtype=torch.int32, device=dev)
    cap = int(b.q_len.sum() + b.t_len.sum() + 16)
    cig = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
    cm = cmoff = None
    if colmax:
        flags |= gsw.GSW_COLMAX
        off = np.zeros(n, np.int64)
        if n:
            off[1:] = np.cumsum(b.t_len.astype(np.int64))[:-1]
        cmoff = T(off)
        cm = torch.zeros(max(int(b.t_len.sum()), 1), dtype=torch.int32, device=dev)
    rc = gsw.gsw_align_batch(ctx.handle, n, q, qo, ql, t, to, tl, b.W, b.gap_open, b.gap_extend, flags,
                             mask_len, res, cig, cap, cm, cmoff, stream=stream)
    torch.cuda.synchronize()
    assert rc == gsw.GSW_OK
    r = res.cpu().numpy().view(gsw.RESULT_DTYPE)
    out_cm = (cm.cpu().numpy(), off) if colmax else (None, None)
    return r, cig.cpu().numpy().view(np.uint32), out_cm


def gpu_cigar(res, cig, p):
    n = int(res["cigar_len"][p])
    o = int(res["cigar_off"][p])
    if n <= 0:
        return []
    return oracle.decode_cigar(cig[o:o + n])


def compare(b, ora, got, check_begin=True, check_cigar=True, check_colmax=True, idx=None):
    """Asserts equality; returns the number of pairs compared."""
    ores, ocg, ocm = ora
    gres, gcig, (gcm, gcmoff) = got
    pairs = range(b.npairs) if idx is None else idx
    bad = []
    for p in pairs:
        fields = FIELDS if check_begin else tuple(f for f in FIELDS if "begin" not in f)
        for f in fields:
            if int(ores[f][p]) != int(gres[f][p]):
                bad.append((p, f, int(ores[f][p]), int(gres[f][p])))
        if gres["flags"][p] & 0x80:
            bad.append((p, "internal-flag", 0, int(gres["flags"][p])))
        if check_cigar:
            want = oracle.decode_cigar(ocg[p, : ores["cigar_len"][p]])
            have = gpu_cigar(gres, gcig, p)
            if want != have:
                bad.append((p, "cigar", oracle.cigar_string(want), oracle.cigar_string(have)))
        if check_colmax and gcm is not None:
            cm, cmoff = ocm
            a = cm[cmoff[p]: cmoff[p] + b.t_len[p]]
            c = gcm[gcmoff[p]: gcmoff[p] + b.t_len[p]]
            if not np.array_equal(a, c):
                j = int(np.nonzero(a != c)[0][0])
                bad.append((p, f"colmax[{j}]", int(a[j]), int(c[j])))
        if len(bad) > 20:
            break
    assert not bad, f"{len(bad)} mismatches, first: {bad[:10]}"
    return len(pairs)
