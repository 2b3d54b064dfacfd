"""CPU oracle for the SSW method (Zhao et al. 2012) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, full-matrix int32 restatement of what the method computes
(`gsw_oracle.c`, compiled with gcc into `oracle/_build/`).  Only the tests, the
smoke check and the benchmark's CPU-baseline / reference legs may import this
package.  The product library (`paper_1208_6350_gb300`) never imports it and
shares no code with it.

Functions and the passages they follow:
  fill       local SW-Gotoh fill, the per-column "max" array and the end cell
             (Algorithm and implementation, item (1); Fig. 1 caption)
  secondary  masked second-best from the max array (item (2); Fig. 1 caption)
  begin      reversed SW from the end (item (1); Fig. 1 caption)
  cigar      global Gotoh between begin and end with traceback (item (1))
  align      all four for one pair; align_batch for many pairs on all cores
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgsw_oracle.so")
_lock = threading.Lock()
_lib = None

OP_M, OP_I, OP_D = 0, 1, 2
OP_CHARS = "MID"


class OraResult(ctypes.Structure):
    _fields_ = [
        ("score1", ctypes.c_int32),
        ("score2", ctypes.c_int32),
        ("ref_begin1", ctypes.c_int32),
        ("ref_end1", ctypes.c_int32),
        ("read_begin1", ctypes.c_int32),
        ("read_end1", ctypes.c_int32),
        ("ref_end2", ctypes.c_int32),
        ("cigar_len", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]


RESULT_DTYPE = np.dtype([(name, np.int32) for name, _ in OraResult._fields_])


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, portable flags only)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-fPIC",
                        "-shared", "-pthread", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32 = ctypes.c_int32
    lib.ora_fill.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, P, P, P]
    lib.ora_secondary.argtypes = [P, i32, i32, i32, P, P]
    lib.ora_begin.argtypes = [P, P, P, i32, i32, i32, i32, i32, i32, P, P]
    lib.ora_cigar.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, i32, P, P]
    lib.ora_align.argtypes = [P, i32, P, i32, P, i32, i32, i32, i32, P, P, i32,
                              ctypes.POINTER(OraResult)]
    lib.ora_align_batch.argtypes = [i32, P, P, P, P, P, P, P, i32, i32, i32, i32, P, P, i32,
                                    P, P, i32]
    for f in (lib.ora_fill, lib.ora_secondary, lib.ora_begin, lib.ora_cigar, lib.ora_align,
              lib.ora_align_batch):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _mat(W):
    W = np.ascontiguousarray(np.asarray(W, dtype=np.int8))
    assert W.ndim == 2 and W.shape[0] == W.shape[1]
    return W


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def fill(q, t, W, gap_open, gap_extend):
    """Local fill: returns (colmax[n], score1, end_t, end_q)."""
    lib = _load()
    q, t, W = _u8(q), _u8(t), _mat(W)
    cm = np.zeros(max(len(t), 1), dtype=np.int32)
    s, et, eq = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.ora_fill(_ptr(q), len(q), _ptr(t), len(t), _ptr(W), W.shape[0], gap_open,
                        gap_extend, _ptr(cm), ctypes.byref(s), ctypes.byref(et),
                        ctypes.byref(eq)), "ora_fill")
    return cm[:len(t)], s.value, et.value, eq.value


def secondary(colmax, end_t, mask_len):
    lib = _load()
    cm = np.ascontiguousarray(np.asarray(colmax, dtype=np.int32))
    s2, e2 = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.ora_secondary(_ptr(cm), len(cm), end_t, mask_len, ctypes.byref(s2),
                             ctypes.byref(e2)), "ora_secondary")
    return s2.value, e2.value


def begin(q, t, W, gap_open, gap_extend, end_q, end_t, score1):
    lib = _load()
    q, t, W = _u8(q), _u8(t), _mat(W)
    bq, bt = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.ora_begin(_ptr(q), _ptr(t), _ptr(W), W.shape[0], gap_open, gap_extend, end_q,
                         end_t, score1, ctypes.byref(bq), ctypes.byref(bt)), "ora_begin")
    return bq.value, bt.value


def cigar(qs, ts, W, gap_open, gap_extend, cap=None):
    """Global alignment of qs x ts: returns (list of (len, op) runs, score)."""
    lib = _load()
    qs, ts, W = _u8(qs), _u8(ts), _mat(W)
    cap = cap if cap is not None else len(qs) + len(ts) + 1
    buf = np.zeros(max(cap, 1), dtype=np.uint32)
    n, sc = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.ora_cigar(_ptr(qs), len(qs), _ptr(ts), len(ts), _ptr(W), W.shape[0], gap_open,
                         gap_extend, _ptr(buf), cap, ctypes.byref(n), ctypes.byref(sc)),
           "ora_cigar")
    return decode_cigar(buf[:n.value]), sc.value


def decode_cigar(words):
    return [(int(w) >> 4, int(w) & 15) for w in words]


def cigar_string(runs):
    return "".join(f"{n}{OP_CHARS[op]}" for n, op in runs)


def align(q, t, W, gap_open, gap_extend, mask_len=-1):
    """All outputs for one pair as a dict (score1, score2, ends, begins, cigar, colmax)."""
    lib = _load()
    q, t, W = _u8(q), _u8(t), _mat(W)
    cap = len(q) + len(t) + 1
    buf = np.zeros(cap, dtype=np.uint32)
    cm = np.zeros(max(len(t), 1), dtype=np.int32)
    r = OraResult()
    _check(lib.ora_align(_ptr(q), len(q), _ptr(t), len(t), _ptr(W), W.shape[0], gap_open,
                         gap_extend, mask_len, _ptr(cm), _ptr(buf), cap, ctypes.byref(r)),
           "ora_align")
    out = {name: getattr(r, name) for name, _ in OraResult._fields_}
    out["cigar"] = decode_cigar(buf[:r.cigar_len])
    out["colmax"] = cm[:len(t)].copy()
    return out


def align_batch(qa, qoff, qlen, ta, toff, tlen, W, gap_open, gap_extend, mask_len=-1,
                nthreads=None, cigar_stride=0, colmax=False):
    """Aligns pairs (query p = qa[qoff[p]:qoff[p]+qlen[p]], same for targets).

    Returns (results structured array, cigar words [npairs, cigar_stride] or None,
    colmax flat array and its per-pair offsets, or None)."""
    lib = _load()
    qa, ta, W = _u8(qa), _u8(ta), _mat(W)
    qoff = np.ascontiguousarray(qoff, dtype=np.int64)
    toff = np.ascontiguousarray(toff, dtype=np.int64)
    qlen = np.ascontiguousarray(qlen, dtype=np.int32)
    tlen = np.ascontiguousarray(tlen, dtype=np.int32)
    npairs = len(qlen)
    res = np.zeros(npairs, dtype=RESULT_DTYPE)
    cg = np.zeros((npairs, cigar_stride), dtype=np.uint32) if cigar_stride > 0 else None
    cm = cmoff = None
    if colmax:
        cmoff = np.zeros(npairs, dtype=np.int64)
        if npairs:
            cmoff[1:] = np.cumsum(tlen.astype(np.int64))[:-1]
        cm = np.zeros(max(int(tlen.sum()), 1), dtype=np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib.ora_align_batch(npairs, _ptr(qa), _ptr(qoff), _ptr(qlen), _ptr(ta), _ptr(toff),
                        _ptr(tlen), _ptr(W), W.shape[0], gap_open, gap_extend, mask_len,
                        _ptr(res), _ptr(cg), cigar_stride, _ptr(cm), _ptr(cmoff), nthreads)
    return res, cg, (cm, cmoff) if colmax else None
