"""CPU checks of the boundary: the library builds, loads and exports every
function include/gsw.h declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1208_6350_gb300 import _build, gsw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("gsw.h",):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gsw_\w+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    lib = ctypes.CDLL(_build.build())
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/gsw.h but not exported"


def test_strerror_and_version_need_no_gpu():
    assert gsw.strerror(gsw.GSW_EINVAL) == "invalid argument"
    assert gsw.strerror(gsw.GSW_ECIGAR_SPACE) == "CIGAR buffer too small"
    assert "sm_103a" in gsw.gsw_version()


def test_result_record_layout():
    assert gsw.RESULT_DTYPE.itemsize == 48
    assert gsw.RESULT_DTYPE.fields["cigar_off"][1] == 32


def test_null_context_rejected_without_gpu():
    import numpy as np
    W = np.eye(4, dtype=np.int8)
    rc = gsw.load().gsw_align_batch(None, 1, None, None, None, None, None, None,
                                    W.ctypes.data, 4, 3, 1, 0, -1, None, None, 0, None, None, None)
    assert rc == gsw.GSW_EINVAL


def test_bad_scoring_rejected_without_gpu():
    import numpy as np
    W = np.eye(4, dtype=np.int8)
    lib = gsw.load()
    # gap_extend > gap_open is rejected before any device work
    rc = lib.gsw_align_batch(None, 1, None, None, None, None, None, None, W.ctypes.data, 4, 1, 3, 0,
                             -1, None, None, 0, None, None, None)
    assert rc == gsw.GSW_EINVAL
    rc = lib.gsw_align_batch(None, 1, None, None, None, None, None, None, W.ctypes.data, 40, 3, 1,
                             0, -1, None, None, 0, None, None, None)
    assert rc == gsw.GSW_EINVAL


def test_tuning_calls_reject_null_context_without_gpu():
    lib = gsw.load()
    assert lib.gsw_context_set_tune(None, None) == gsw.GSW_EINVAL
    assert lib.gsw_autotune(None, None, 4, 3, 1, 1000, None) == gsw.GSW_EINVAL


def test_pack2_layout_and_packed_flag_checks_without_gpu():
    import numpy as np
    rng = np.random.default_rng(3)
    c = rng.integers(0, 4, 1003).astype(np.uint8)
    p = gsw.pack2(c)
    assert len(p) == 251
    back = np.array([(p[x // 4] >> (2 * (x % 4))) & 3 for x in range(len(c))], np.uint8)
    assert (back == c).all()
    W = np.eye(20, dtype=np.int8)
    lib = gsw.load()
    # packed input needs the 4-letter alphabet: rejected before any device work
    rc = lib.gsw_align_batch(None, 1, None, None, None, None, None, None, W.ctypes.data, 20, 3, 1,
                             gsw.GSW_PACKED2, -1, None, None, 0, None, None, None)
    assert rc == gsw.GSW_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    # a fresh interpreter whose library path points nowhere: load() raises
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1208_6350_gb300 import _build, gsw\n"
        "_build.LIB = %r\n"
        "try:\n"
        "    gsw.load(build_if_missing=False)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('loaded')\n" % (ROOT, str(tmp_path / "absent" / "libgsw.so")))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised: CUDA library not built"), out.stdout


def test_context_without_a_gpu_raises():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gsw.GswError):
        gsw.Context(0, 1 << 20)


def test_library_is_rebuilt_when_the_nvcc_flags_change(monkeypatch):
    _build.build()
    assert _build.up_to_date()
    monkeypatch.setenv("GSW_NVCC_EXTRA", "-DGSW_FLAG_STAMP_CHECK=1")
    assert not _build.up_to_date()
    monkeypatch.delenv("GSW_NVCC_EXTRA")
    assert _build.up_to_date()


def test_pair_cigar_and_cigar_string():
    rec = np.zeros(3, gsw.RESULT_DTYPE)
    words = np.array([7, 7, (3 << 4) | 0, (1 << 4) | 2, (2 << 4) | 0, (4 << 4) | 1], np.uint32)
    rec[0]["cigar_off"], rec[0]["cigar_len"] = 2, 4
    rec[2]["cigar_len"], rec[2]["flags"] = -9, gsw.GSW_RES_CIGAR_SPACE
    runs = gsw.pair_cigar(rec[0], words)
    assert runs == [(3, 0), (1, 2), (2, 0), (4, 1)]
    assert gsw.cigar_string(runs) == "3M1D2M4I"
    assert gsw.pair_cigar(rec[1], words) == []           # no CIGAR
    with pytest.raises(ValueError, match="needs 9 words"):
        gsw.pair_cigar(rec[2], words)
    # int32 buffers (torch's dtype for the device copy) read the same
    assert gsw.pair_cigar(rec[0], words.view(np.int32)) == runs


def _header_defines():
    src = open(os.path.join(ROOT, "include", "gsw.h")).read()
    out = {}
    for name, val in re.findall(r"#define\s+(GSW_\w+)\s+\(?(-?(?:0x)?[0-9a-fA-F]+)u?\)?", src):
        out[name] = int(val, 0)
    return out


def test_binding_constants_match_the_header():
    d = _header_defines()
    for name in ("GSW_OK", "GSW_EINVAL", "GSW_ENOMEM", "GSW_ECUDA", "GSW_ETIMEDOUT", "GSW_ECIGAR_SPACE",
                 "GSW_EOVERFLOW", "GSW_ENOTFOUND", "GSW_ESTATE", "GSW_EINTERNAL", "GSW_BEGIN", "GSW_CIGAR",
                 "GSW_COLMAX", "GSW_HOST_IO", "GSW_FORCE_S32", "GSW_PLAIN", "GSW_TIMING", "GSW_PACKED2",
                 "GSW_RES_S32", "GSW_RES_CIGAR_SPACE", "GSW_RES_INVALID", "GSW_RES_INTERNAL",
                 "GSW_STATIC_MAX_TARGET"):
        assert getattr(gsw, name) == d[name], name


def test_every_error_code_has_a_name():
    names = {gsw.strerror(c) for c in range(0, -10, -1)}
    assert len(names) == 10 and "unknown error" not in names
    assert gsw.strerror(gsw.GSW_EINTERNAL) == "internal consistency check failed"


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes mirrors of gsw_stats and gsw_record against gcc's layout of
    include/gsw.h."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "lay.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gsw.h"\n'
        'int main(void) {\n'
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(gsw_stats), offsetof(gsw_stats, ring_words),'
        ' offsetof(gsw_stats, internal_pairs), sizeof(gsw_record), offsetof(gsw_record, colmax));\n'
        ' printf("%zu %zu %zu %zu\\n", sizeof(gsw_result), sizeof(gsw_serve_config), sizeof(gsw_serve_stats),'
        ' offsetof(gsw_serve_stats, graph_batches));\n return 0; }\n')
    exe = tmp_path / "lay"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    a = [int(x) for x in a.split()]
    b = [int(x) for x in b.split()]
    assert a == [ctypes.sizeof(gsw.GswStats), gsw.GswStats.ring_words.offset, gsw.GswStats.internal_pairs.offset,
                 ctypes.sizeof(gsw.GswRecord), gsw.GswRecord.colmax.offset]
    assert b == [gsw.RESULT_DTYPE.itemsize, ctypes.sizeof(gsw.ServeConfig), ctypes.sizeof(gsw.ServeStats),
                 gsw.ServeStats.graph_batches.offset]


def test_results_handle_calls_check_arguments_without_gpu():
    lib = gsw.load()
    assert lib.gsw_results_count(None) == 0
    rec = gsw.GswRecord()
    assert lib.gsw_results_get(None, 0, ctypes.byref(rec)) == gsw.GSW_EINVAL
    lib.gsw_results_free(None)  # ignored
    W = np.eye(4, dtype=np.int8)
    out = ctypes.c_void_p()
    rc = lib.gsw_align_batch_results(None, 1, None, None, None, None, None, None, W.ctypes.data, 4, 3, 1, 0, -1,
                                     None, ctypes.byref(out))
    assert rc == gsw.GSW_EINVAL and out.value is None
    assert lib.gsw_align_batch_results(None, 1, None, None, None, None, None, None, W.ctypes.data, 4, 3, 1, 0,
                                       -1, None, None) == gsw.GSW_EINVAL
    assert lib.gsw_serve_poll_results(None, 1, 0, ctypes.byref(out)) == gsw.GSW_EINVAL


def test_static_fill_checks_arguments_before_any_device_work():
    W = np.eye(4, dtype=np.int8)
    lib = gsw.load()
    # flags other than GSW_COLMAX, a too-large mask, O < X, a NULL pointer
    assert lib.gsw_fill_static(1, None, None, None, None, None, None, 10, W.ctypes.data, 4, 3, 1,
                               gsw.GSW_CIGAR, -1, None, None, None, None) == gsw.GSW_EINVAL
    assert lib.gsw_fill_static(1, None, None, None, None, None, None, 10, W.ctypes.data, 4, 3, 1, 0,
                               (1 << 30) + 1, None, None, None, None) == gsw.GSW_EINVAL
    assert lib.gsw_fill_static(1, None, None, None, None, None, None, 10, W.ctypes.data, 4, 1, 3, 0, -1,
                               None, None, None, None) == gsw.GSW_EINVAL
    assert "gap" in gsw.last_error()
    assert lib.gsw_fill_static(1, None, None, None, None, None, None, 10, W.ctypes.data, 4, 3, 1, 0, -1,
                               None, None, None, None) == gsw.GSW_EINVAL
    assert "NULL" in gsw.last_error()
    # a maximum target length beyond the static slot's
    assert lib.gsw_fill_static(1, 1, 1, 1, 1, 1, 1, gsw.GSW_STATIC_MAX_TARGET + 1, W.ctypes.data, 4, 3, 1, 0, -1,
                               1, None, None, None) == gsw.GSW_EINVAL
    assert "max_target_len" in gsw.last_error()
