"""The C-ABI library builds, loads and exports every entry point of include/dualip.h.

No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dualip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dualip_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libdualip():
    from paper_2603_04621_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dualip_create", "dualip_dual_grad", "dualip_solve", "dualip_destroy",
                     "dualip_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libdualip):
    missing = [n for n in _declared() if not hasattr(libdualip, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2603_04621_gb300 as d

    assert sorted(d.EXPORTS) == _declared()


def _prototypes():
    """name -> parameter count of every function declared in the header."""
    src = open(os.path.join(ROOT, "include", "dualip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(dualip_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argtypes_match_the_prototypes():
    import paper_2603_04621_gb300 as d

    L = d.lib()
    protos = _prototypes()
    assert sorted(protos) == _declared()
    for name, n in protos.items():
        assert len(getattr(L, name).argtypes) == n, name


def test_last_error_is_empty_string_initially(libdualip):
    libdualip.dualip_last_error.restype = ctypes.c_char_p
    assert libdualip.dualip_last_error() == b""


def test_create_rejects_bad_desc_without_a_gpu(libdualip):
    """Argument validation happens before any CUDA call."""
    import paper_2603_04621_gb300 as d

    lib = d.lib()
    h = ctypes.c_void_p()
    assert lib.dualip_create(None, None, ctypes.byref(h)) == d.DUALIP_EINVAL
    desc = d.ProblemDesc(-1, 0, 5, None, None, None, None, None, 0, 0, 0)
    assert lib.dualip_create(ctypes.byref(desc), None, ctypes.byref(h)) == d.DUALIP_EINVAL
    assert b"I >= 0" in lib.dualip_last_error()
    import numpy as np

    off = np.array([0, 2, 1], dtype=np.int64)  # decreasing
    b = np.zeros(3, dtype=np.float32)
    desc = d.ProblemDesc(2, 1, 3, off.ctypes.data, 1, 1, 1, b.ctypes.data, 0, 0, 0)
    assert lib.dualip_create(ctypes.byref(desc), None, ctypes.byref(h)) == d.DUALIP_EINVAL
    assert b"nondecreasing" in lib.dualip_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libdualip.so the binding raises."""
    import paper_2603_04621_gb300 as d

    monkeypatch.setattr(d, "_lib", None)
    monkeypatch.setattr(d, "LIB_PATH", str(tmp_path / "libdualip.so"))
    with pytest.raises(RuntimeError, match="missing"):
        d.lib()


def test_host_argument_checks_of_the_forms(libdualip):
    """Batch and server entry points reject bad arguments before any CUDA call."""
    import paper_2603_04621_gb300 as d

    lib = d.lib()
    out = ctypes.c_void_p()
    assert lib.dualip_batch_create(0, None, ctypes.byref(out)) == d.DUALIP_EINVAL
    assert lib.dualip_server_create(None, ctypes.byref(out)) == d.DUALIP_EINVAL
    bad = d.ServerOpts(0, 4, 10)
    assert lib.dualip_server_create(ctypes.byref(bad), ctypes.byref(out)) == d.DUALIP_EINVAL
    bad = d.ServerOpts(1 << 30, 0, 10)
    assert lib.dualip_server_create(ctypes.byref(bad), ctypes.byref(out)) == d.DUALIP_EINVAL
