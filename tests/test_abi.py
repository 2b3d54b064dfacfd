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
