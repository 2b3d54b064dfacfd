"""Python binding of the C ABI in include/gsw.h (argument marshalling only).

Every function here forwards to libgsw.so, the CUDA library built from
csrc/.  There is no fallback: if the library is missing the calls raise.
PyTorch tensors (device memory, streams) and numpy arrays (host memory, with
GSW_HOST_IO) are accepted wherever the C call takes a pointer.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

GSW_OK = 0
GSW_EINVAL = -1
GSW_ENOMEM = -2
GSW_ECUDA = -3
GSW_ETIMEDOUT = -4
GSW_ECIGAR_SPACE = -5
GSW_EOVERFLOW = -6
GSW_ENOTFOUND = -7
GSW_ESTATE = -8
GSW_EINTERNAL = -9

GSW_BEGIN = 0x1
GSW_CIGAR = 0x2
GSW_COLMAX = 0x4
GSW_HOST_IO = 0x8
GSW_FORCE_S32 = 0x10
GSW_PLAIN = 0x20
GSW_TIMING = 0x40
GSW_PACKED2 = 0x80
GSW_NSTAGES = 7
STAGE_NAMES = ("plan_fwd", "fill_fwd", "refill_s32", "reverse_wide", "band", "trace_wide", "pipeline")

GSW_RES_S32 = 0x1
GSW_RES_CIGAR_SPACE = 0x2
GSW_RES_INVALID = 0x4
GSW_RES_INTERNAL = 0x80

RESULT_DTYPE = np.dtype([
    ("score1", np.int32), ("score2", np.int32), ("ref_begin1", np.int32), ("ref_end1", np.int32),
    ("read_begin1", np.int32), ("read_end1", np.int32), ("ref_end2", np.int32),
    ("cigar_len", np.int32), ("cigar_off", np.int64), ("flags", np.int32), ("reserved", np.int32),
])
assert RESULT_DTYPE.itemsize == 48

_lib = None


class GswStats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int32), ("timed", ctypes.c_int32),
                ("stage_ms", ctypes.c_float * 8), ("graph_segments", ctypes.c_int32),
                ("cigar_words", ctypes.c_int64), ("ring_words", ctypes.c_int64),
                ("ring_pool_words", ctypes.c_int64), ("ring_groups", ctypes.c_int32),
                ("internal_pairs", ctypes.c_int32)]


class GswRecord(ctypes.Structure):
    """One record of a library-owned results handle (gsw_results_get)."""
    _fields_ = [("score1", ctypes.c_int32), ("score2", ctypes.c_int32), ("ref_begin1", ctypes.c_int32),
                ("ref_end1", ctypes.c_int32), ("read_begin1", ctypes.c_int32), ("read_end1", ctypes.c_int32),
                ("ref_end2", ctypes.c_int32), ("lane_bits_used", ctypes.c_uint8),
                ("cigar", ctypes.POINTER(ctypes.c_uint32)), ("cigar_len", ctypes.c_int32),
                ("colmax", ctypes.POINTER(ctypes.c_int32)), ("n", ctypes.c_int32), ("flags", ctypes.c_int32)]


TUNE_BUCKETS = 32
TUNE_ROWS = 32


class GswTune(ctypes.Structure):
    _fields_ = [("fill_class", ctypes.c_int8 * TUNE_BUCKETS), ("gcups", ctypes.c_float * TUNE_BUCKETS),
                ("gcups_default", ctypes.c_float * TUNE_BUCKETS)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("workers", ctypes.c_int32), ("max_batch_pairs", ctypes.c_int32),
                ("max_batch_letters", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_queue_requests", ctypes.c_int32), ("flags", ctypes.c_uint32), ("mask_len", ctypes.c_int32),
                ("matrix", ctypes.c_void_p), ("alphabet", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("heavy_workers", ctypes.c_int32), ("heavy_cells", ctypes.c_int64),
                ("heavy_sm_limit", ctypes.c_int32), ("light_graphs", ctypes.c_int32)]


class ServeTimes(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_double), ("started", ctypes.c_double), ("done", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("pairs", ctypes.c_uint64), ("cells", ctypes.c_uint64), ("busy_seconds", ctypes.c_double),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("graph_batches", ctypes.c_uint64)]


class GswError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}): {last_error()}")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgsw.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.gsw_context_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(P)]
    lib.gsw_context_destroy.argtypes = [P]
    lib.gsw_context_set_sm_limit.argtypes = [P, ctypes.c_int]
    lib.gsw_context_set_sm_limit.restype = ctypes.c_int
    lib.gsw_align_to_reference.argtypes = [P, i32, P, P, P, P, i64, P, i32, i32, i32, u32, i32, i64, P, P, i64, P]
    lib.gsw_align_to_reference.restype = ctypes.c_int
    lib.gsw_align_all_pairs.argtypes = [P, i32, P, P, P, P, i32, i32, i32, u32, i32, i64, P, P, i64, P]
    lib.gsw_align_all_pairs.restype = ctypes.c_int
    lib.gsw_autotune.argtypes = [P, P, i32, i32, i32, i32, ctypes.POINTER(GswTune)]
    lib.gsw_autotune.restype = ctypes.c_int
    lib.gsw_context_set_tune.argtypes = [P, ctypes.POINTER(GswTune)]
    lib.gsw_context_set_tune.restype = ctypes.c_int
    lib.gsw_align_batch.argtypes = [P, i32, P, P, P, P, P, P, P, i32, i32, i32, u32, i32, P, P, i64, P,
                                    P, P]
    lib.gsw_profile_create.argtypes = [P, P, i32, P, i32, i32, i32, ctypes.POINTER(P)]
    lib.gsw_profile_destroy.argtypes = [P]
    lib.gsw_align_profile.argtypes = [P, P, i32, P, P, P, u32, i32, P, P, i64, P, P, P]
    for f in (lib.gsw_context_create, lib.gsw_context_destroy, lib.gsw_align_batch,
              lib.gsw_profile_create, lib.gsw_profile_destroy, lib.gsw_align_profile):
        f.restype = ctypes.c_int
    lib.gsw_align_batch_results.argtypes = [P, i32, P, P, P, P, P, P, P, i32, i32, i32, u32, i32, P,
                                            ctypes.POINTER(P)]
    lib.gsw_align_batch_results.restype = ctypes.c_int
    lib.gsw_results_count.argtypes = [P]
    lib.gsw_results_count.restype = i32
    lib.gsw_results_get.argtypes = [P, i32, ctypes.POINTER(GswRecord)]
    lib.gsw_results_get.restype = ctypes.c_int
    lib.gsw_results_free.argtypes = [P]
    lib.gsw_results_free.restype = None
    lib.gsw_serve_poll_results.argtypes = [P, ctypes.c_uint64, i32, ctypes.POINTER(P)]
    lib.gsw_serve_poll_results.restype = ctypes.c_int
    lib.gsw_fill_static.argtypes = [i32, P, P, P, P, P, P, i32, P, i32, i32, i32, u32, i32, P, P, P, P]
    lib.gsw_fill_static.restype = ctypes.c_int
    lib.gsw_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(P)]
    lib.gsw_serve_destroy.argtypes = [P]
    lib.gsw_serve_submit.argtypes = [P, i32, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.gsw_serve_poll.argtypes = [P, ctypes.c_uint64, i32, P, P, i64, ctypes.POINTER(ctypes.c_int64)]
    lib.gsw_serve_poll_timed.argtypes = [P, ctypes.c_uint64, i32, P, P, i64, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ServeTimes)]
    lib.gsw_serve_get_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
    for f in (lib.gsw_serve_create, lib.gsw_serve_destroy, lib.gsw_serve_submit, lib.gsw_serve_poll,
              lib.gsw_serve_poll_timed, lib.gsw_serve_get_stats):
        f.restype = ctypes.c_int
    lib.gsw_serve_now.argtypes = [P]
    lib.gsw_serve_now.restype = ctypes.c_double
    lib.gsw_last_stats.argtypes = [P, ctypes.POINTER(GswStats)]
    lib.gsw_last_stats.restype = ctypes.c_int
    lib.gsw_strerror.argtypes = [ctypes.c_int]
    lib.gsw_strerror.restype = ctypes.c_char_p
    lib.gsw_last_error.restype = ctypes.c_char_p
    lib.gsw_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().gsw_strerror(code).decode()


def last_error() -> str:
    return load().gsw_last_error().decode()


def gsw_version() -> str:
    return load().gsw_version().decode()


def _ptr(x):
    """Address of a torch tensor, numpy array, or an int; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(rc, what):
    if rc != GSW_OK:
        raise GswError(rc, what)
    return rc


def gsw_context_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().gsw_context_create(device, mem_budget_bytes, ctypes.byref(out)), "gsw_context_create")
    return out.value


def gsw_context_destroy(ctx: int) -> None:
    _check(load().gsw_context_destroy(ctx), "gsw_context_destroy")


def gsw_align_to_reference(ctx, nreads, q, q_off, q_len, ref, ref_len, matrix, gap_open, gap_extend,
                           flags=GSW_CIGAR, mask_len=-1, window=0, results=None, cigar=None, cigar_capacity=0,
                           stream=None, check=True) -> int:
    """Direct call of gsw_align_to_reference; pointer arguments may be tensors/arrays."""
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    rc = load().gsw_align_to_reference(ctx, nreads, _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(ref), ref_len,
                                       m.ctypes.data, m.shape[0], gap_open, gap_extend, flags, mask_len, window,
                                       _ptr(results), _ptr(cigar), cigar_capacity, _stream_handle(stream))
    if check and rc != GSW_ECIGAR_SPACE:
        _check(rc, "gsw_align_to_reference")
    return rc


def gsw_align_batch(ctx, npairs, q, q_off, q_len, t, t_off, t_len, matrix, gap_open, gap_extend,
                    flags=0, mask_len=-1, results=None, cigar=None, cigar_capacity=0, colmax=None,
                    colmax_off=None, stream=None, check=True) -> int:
    """Direct call of gsw_align_batch; pointer arguments may be tensors/arrays."""
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    A = m.shape[0]
    st = _stream_handle(stream)
    rc = load().gsw_align_batch(ctx, npairs, _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(t), _ptr(t_off),
                                _ptr(t_len), m.ctypes.data, A, gap_open, gap_extend, flags, mask_len,
                                _ptr(results), _ptr(cigar), cigar_capacity, _ptr(colmax),
                                _ptr(colmax_off), st)
    if check and rc != GSW_ECIGAR_SPACE:
        _check(rc, "gsw_align_batch")
    return rc


def gsw_last_stats(ctx) -> dict:
    st = GswStats()
    _check(load().gsw_last_stats(ctx, ctypes.byref(st)), "gsw_last_stats")
    out = {"kernel_launches": st.kernel_launches, "timed": bool(st.timed), "graph_segments": st.graph_segments,
           "cigar_words": st.cigar_words, "ring_words": st.ring_words, "ring_pool_words": st.ring_pool_words,
           "ring_groups": st.ring_groups, "internal_pairs": st.internal_pairs}
    if st.timed:
        out["stage_ms"] = {n: float(st.stage_ms[k]) for k, n in enumerate(STAGE_NAMES)}
    return out


def gsw_align_batch_results(ctx, npairs, q, q_off, q_len, t, t_off, t_len, matrix, gap_open, gap_extend,
                            flags=0, mask_len=-1, stream=None):
    """gsw_align_batch_results; returns (status, handle) -- the handle (an int)
    is set on GSW_OK and GSW_EINTERNAL and must go to gsw_results_free."""
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    out = ctypes.c_void_p()
    rc = load().gsw_align_batch_results(ctx, npairs, _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(t), _ptr(t_off),
                                        _ptr(t_len), m.ctypes.data, m.shape[0], gap_open, gap_extend, flags,
                                        mask_len, _stream_handle(stream), ctypes.byref(out))
    return rc, out.value


def gsw_results_count(handle) -> int:
    return load().gsw_results_count(handle)


def gsw_results_get(handle, i) -> dict:
    """Record i of a results handle as a dict (CIGAR as (length, op) runs,
    the max array as a numpy copy, or None)."""
    r = GswRecord()
    _check(load().gsw_results_get(handle, i, ctypes.byref(r)), "gsw_results_get")
    out = {k: getattr(r, k) for k, _ in GswRecord._fields_ if k not in ("cigar", "colmax")}
    out["cigar"] = [(int(r.cigar[k]) >> 4, int(r.cigar[k]) & 15) for k in range(max(r.cigar_len, 0))] \
        if r.cigar else []
    out["colmax"] = np.ctypeslib.as_array(r.colmax, shape=(r.n,)).copy() if r.colmax and r.n > 0 else None
    return out


def gsw_results_free(handle) -> None:
    load().gsw_results_free(handle)


GSW_STATIC_MAX_TARGET = 1024


def gsw_fill_static(npairs, q, q_off, q_len, t, t_off, t_len, max_target_len, matrix, gap_open,
                    gap_extend, flags=0, mask_len=-1, results=None, colmax=None, colmax_off=None,
                    stream=None) -> int:
    """Allocation-free forward fill (device pointers only); returns the status code."""
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    return load().gsw_fill_static(npairs, _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(t), _ptr(t_off),
                                  _ptr(t_len), max_target_len, m.ctypes.data, m.shape[0], gap_open,
                                  gap_extend, flags, mask_len, _ptr(results), _ptr(colmax),
                                  _ptr(colmax_off), _stream_handle(stream))


def gsw_profile_create(ctx, query, matrix, gap_open, gap_extend) -> int:
    q = np.ascontiguousarray(query, dtype=np.uint8)
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    out = ctypes.c_void_p()
    _check(load().gsw_profile_create(ctx, q.ctypes.data, len(q), m.ctypes.data, m.shape[0], gap_open,
                                     gap_extend, ctypes.byref(out)), "gsw_profile_create")
    return out.value


def gsw_profile_destroy(prof) -> None:
    _check(load().gsw_profile_destroy(prof), "gsw_profile_destroy")


def gsw_align_profile(ctx, prof, ntargets, t, t_off, t_len, flags=0, mask_len=-1, results=None,
                      cigar=None, cigar_capacity=0, colmax=None, colmax_off=None, stream=None,
                      check=True) -> int:
    rc = load().gsw_align_profile(ctx, prof, ntargets, _ptr(t), _ptr(t_off), _ptr(t_len), flags,
                                  mask_len, _ptr(results), _ptr(cigar), cigar_capacity, _ptr(colmax),
                                  _ptr(colmax_off), _stream_handle(stream))
    if check and rc != GSW_ECIGAR_SPACE:
        _check(rc, "gsw_align_profile")
    return rc


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


CIGAR_OPS = "MID"  # op codes 0, 1, 2 of a CIGAR word (len << 4) | op


def pair_cigar(record, cigar_words):
    """One pair's CIGAR as (length, op) runs: the words its record points at in
    the batch's CIGAR buffer.  Empty when the pair has no CIGAR; raises when the
    pair's CIGAR did not fit the buffer (GSW_RES_CIGAR_SPACE)."""
    n = int(record["cigar_len"])
    if int(record["flags"]) & GSW_RES_CIGAR_SPACE:
        raise ValueError(f"the pair's CIGAR did not fit the buffer: it needs {-n} words")
    if n <= 0:
        return []
    off = int(record["cigar_off"])
    w = np.asarray(cigar_words[off: off + n]).view(np.uint32)
    return [(int(x) >> 4, int(x) & 15) for x in w]


def cigar_string(runs) -> str:
    """SAM-style text of (length, op) runs, e.g. [(3, 0), (1, 2), (2, 0)] -> "3M1D2M"."""
    return "".join(f"{n}{CIGAR_OPS[op]}" for n, op in runs)


def pack2(codes) -> np.ndarray:
    """DNA codes 0..3 packed 4 to a byte (letter x in bits 2(x%4) of byte x/4),
    the GSW_PACKED2 layout; offsets and lengths stay in letters."""
    c = np.ascontiguousarray(codes, np.uint8)
    n = len(c)
    pad = np.zeros((n + 3) // 4 * 4, np.uint8)
    pad[:n] = c & 3
    p = pad.reshape(-1, 4)
    return (p[:, 0] | (p[:, 1] << 2) | (p[:, 2] << 4) | (p[:, 3] << 6)).astype(np.uint8)


class Context:
    """Owns a gsw context; convenience wrappers over the C calls."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.device = device
        self.handle = gsw_context_create(device, mem_budget_bytes)

    def close(self):
        if self.handle:
            gsw_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, matrix, gap_open, gap_extend, target_len=1000) -> dict:
        """Measures the fill class per query-length bucket (gsw_autotune) and
        installs the fastest; returns {"fill_class", "gcups", "gcups_default"}."""
        m = np.ascontiguousarray(matrix, dtype=np.int8)
        t = GswTune()
        _check(load().gsw_autotune(self.handle, m.ctypes.data, m.shape[0], gap_open, gap_extend, target_len,
                                   ctypes.byref(t)), "gsw_autotune")
        return {"fill_class": list(t.fill_class), "gcups": [round(x, 1) for x in t.gcups],
                "gcups_default": [round(x, 1) for x in t.gcups_default]}

    def set_tune(self, fill_class=None):
        """Installs a class per bucket (-1 default rule, 0..6 group variants, 8
        the CTA kernel); None restores the default rule."""
        if fill_class is None:
            _check(load().gsw_context_set_tune(self.handle, None), "gsw_context_set_tune")
            return
        t = GswTune()
        for b, c in enumerate(fill_class):
            t.fill_class[b] = int(c)
        _check(load().gsw_context_set_tune(self.handle, ctypes.byref(t)), "gsw_context_set_tune")

    def align_all_pairs(self, seq, off, length, matrix, gap_open, gap_extend, flags=0, mask_len=-1, chunk=0,
                        cigar_capacity=None):
        """Every pair i < j of one sequence set (host arrays; gsw_align_all_pairs
        with GSW_HOST_IO); records in row-major triangle order."""
        seq = np.ascontiguousarray(seq, np.uint8)
        off = np.ascontiguousarray(off, np.int64)
        length = np.ascontiguousarray(length, np.int32)
        m = np.ascontiguousarray(matrix, dtype=np.int8)
        n = len(length)
        npairs = n * (n - 1) // 2
        res = np.zeros(npairs, RESULT_DTYPE)
        if cigar_capacity is None:
            cigar_capacity = int(npairs * (2 * int(length.max(initial=0)) + 2)) if flags & GSW_CIGAR else 0
        cig = np.zeros(max(cigar_capacity, 1), np.uint32)
        rc = load().gsw_align_all_pairs(self.handle, n, _ptr(seq), _ptr(off), _ptr(length), m.ctypes.data,
                                        m.shape[0], gap_open, gap_extend, flags | GSW_HOST_IO, mask_len, chunk,
                                        _ptr(res), _ptr(cig), cigar_capacity, None)
        return res, cig, rc

    def align_to_reference(self, q, q_off, q_len, ref, matrix, gap_open, gap_extend, flags=GSW_CIGAR,
                           mask_len=-1, window=0, cigar_capacity=None):
        """Reads (host arrays) against one long reference (gsw_align_to_reference,
        GSW_HOST_IO); returns (records, cigar words, status)."""
        q = np.ascontiguousarray(q, np.uint8)
        ref = np.ascontiguousarray(ref, np.uint8)
        q_off = np.ascontiguousarray(q_off, np.int64)
        q_len = np.ascontiguousarray(q_len, np.int32)
        m = np.ascontiguousarray(matrix, dtype=np.int8)
        n = len(q_len)
        res = np.zeros(n, RESULT_DTYPE)
        if cigar_capacity is None:
            cigar_capacity = int(2 * q_len.sum() + 64 * n + 64) if flags & GSW_CIGAR else 0
        cig = np.zeros(max(cigar_capacity, 1), np.uint32)
        rc = load().gsw_align_to_reference(self.handle, n, _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(ref), len(ref),
                                           m.ctypes.data, m.shape[0], gap_open, gap_extend, flags | GSW_HOST_IO,
                                           mask_len, window, _ptr(res), _ptr(cig), cigar_capacity, None)
        return res, cig, rc

    def align_host(self, q, q_off, q_len, t, t_off, t_len, matrix, gap_open, gap_extend,
                   flags=GSW_CIGAR, mask_len=-1, cigar_capacity=None, colmax=False):
        """Host numpy arrays in, host results out (GSW_HOST_IO)."""
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        q_off = np.ascontiguousarray(q_off, np.int64)
        t_off = np.ascontiguousarray(t_off, np.int64)
        q_len = np.ascontiguousarray(q_len, np.int32)
        t_len = np.ascontiguousarray(t_len, np.int32)
        n = len(q_len)
        res = np.zeros(n, RESULT_DTYPE)
        if cigar_capacity is None:
            cigar_capacity = int(16 * n + 1024) if flags & GSW_CIGAR else 0
        cig = np.zeros(max(cigar_capacity, 1), np.uint32)
        cm = cmoff = None
        if colmax:
            flags |= GSW_COLMAX
            cmoff = np.zeros(n, np.int64)
            if n:
                cmoff[1:] = np.cumsum(t_len.astype(np.int64))[:-1]
            cm = np.zeros(max(int(t_len.sum()), 1), np.int32)
        rc = gsw_align_batch(self.handle, n, q, q_off, q_len, t, t_off, t_len, matrix, gap_open,
                             gap_extend, flags | GSW_HOST_IO, mask_len, res, cig, cigar_capacity, cm,
                             cmoff)
        return res, cig, (cm, cmoff), rc


class Server:
    """Continuous-batching server (gsw_serve_*); host numpy arrays in and out."""

    def __init__(self, matrix, gap_open, gap_extend, flags=GSW_CIGAR, mask_len=-1, device=0, workers=4,
                 max_batch_pairs=8192, max_batch_letters=16 << 20, mem_budget_bytes=8 << 30, heavy_workers=0,
                 heavy_cells=0, heavy_sm_limit=0, light_graphs=0):
        self._m = np.ascontiguousarray(matrix, dtype=np.int8)
        cfg = ServeConfig(device, workers, max_batch_pairs, max_batch_letters, mem_budget_bytes, 0, flags,
                          mask_len, self._m.ctypes.data, self._m.shape[0], gap_open, gap_extend, heavy_workers,
                          heavy_cells, heavy_sm_limit, light_graphs)
        out = ctypes.c_void_p()
        _check(load().gsw_serve_create(ctypes.byref(cfg), ctypes.byref(out)), "gsw_serve_create")
        self.handle = out.value

    def submit(self, q, q_off, q_len, t, t_off, t_len) -> int:
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        q_off = np.ascontiguousarray(q_off, np.int64)
        t_off = np.ascontiguousarray(t_off, np.int64)
        q_len = np.ascontiguousarray(q_len, np.int32)
        t_len = np.ascontiguousarray(t_len, np.int32)
        rid = ctypes.c_uint64()
        _check(load().gsw_serve_submit(self.handle, len(q_len), _ptr(q), _ptr(q_off), _ptr(q_len), _ptr(t),
                                       _ptr(t_off), _ptr(t_len), ctypes.byref(rid)), "gsw_serve_submit")
        return rid.value

    def poll(self, req_id, npairs, timeout_us=-1, cigar_capacity=None, times=False):
        """Returns (status, results, cigar words) -- results None while pending;
        with times=True a fourth item: (submitted, started, done) seconds on
        the server clock."""
        res = np.zeros(npairs, RESULT_DTYPE)
        cap = cigar_capacity if cigar_capacity is not None else 64 * npairs + 64
        cig = np.zeros(max(cap, 1), np.uint32)
        used = ctypes.c_int64()
        tm = ServeTimes()
        rc = load().gsw_serve_poll_timed(self.handle, req_id, timeout_us, _ptr(res), _ptr(cig), cap,
                                         ctypes.byref(used), ctypes.byref(tm))
        if rc == GSW_ECIGAR_SPACE:
            return self.poll(req_id, npairs, timeout_us, int(used.value), times)
        if rc == GSW_ETIMEDOUT:
            return (rc, None, None, None) if times else (rc, None, None)
        out = (rc, res, cig[: used.value])
        return out + ((tm.submitted, tm.started, tm.done),) if times else out

    def poll_results(self, req_id, timeout_us=-1):
        """gsw_serve_poll_results: (status, handle or None); free the handle
        with gsw_results_free."""
        out = ctypes.c_void_p()
        rc = load().gsw_serve_poll_results(self.handle, req_id, timeout_us, ctypes.byref(out))
        return rc, out.value

    def now(self) -> float:
        """The server clock (seconds since creation)."""
        return load().gsw_serve_now(self.handle)

    def stats(self) -> dict:
        st = ServeStats()
        _check(load().gsw_serve_get_stats(self.handle, ctypes.byref(st)), "gsw_serve_get_stats")
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def close(self):
        if self.handle:
            _check(load().gsw_serve_destroy(self.handle), "gsw_serve_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
