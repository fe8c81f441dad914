"""Host-side checks of the C ABI that need no GPU: the library builds/loads,
exports every entry point declared in include/fam.h, and rejects bad
arguments (and an injected allocation failure) before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2609_26194_b300 import fam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fam.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fam_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(fam.LIB_PATH):
        from paper_2609_26194_b300 import build
        build.build()
    return fam.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fam.EXPORTS)


def _grid(d=2, nx=16, ny=16):
    return fam.Grid(d, nx, ny, 0.0, 1.0, 0.0, 1.0)


@pytest.mark.parametrize("kw,expect", [
    (dict(k=2), 1), (dict(k=7), 1), (dict(eq=5), 1), (dict(bc=3), 1), (dict(prec=16), 1),
    (dict(nx=3), 1), (dict(d=3), 1), (dict(gamma=1.0), 1),
])
def test_create_rejects_bad_arguments(L, kw, expect):
    g = _grid(d=kw.get("d", 2), nx=kw.get("nx", 16))
    h = ctypes.c_void_p()
    rc = L.fam_create(ctypes.byref(h), ctypes.byref(g), kw.get("k", 5), kw.get("eq", 2), kw.get("bc", 0),
                      kw.get("gamma", 1.4), kw.get("prec", 64), None)
    assert rc == expect
    assert not h.value


def test_create_null_pointers(L):
    assert L.fam_create(None, None, 5, 2, 0, 1.4, 64, None) == 1
    h = ctypes.c_void_p()
    assert L.fam_create(ctypes.byref(h), None, 5, 2, 0, 1.4, 64, None) == 1


def test_injected_allocation_failure_reports_nomem(L, monkeypatch):
    monkeypatch.setenv("FAM_FAULT_ALLOC", "1")
    g = _grid()
    h = ctypes.c_void_p()
    assert L.fam_create(ctypes.byref(h), ctypes.byref(g), 5, 2, 0, 1.4, 64, None) == 2
    assert not h.value


def test_batch2d_create_rejects_bad_arguments(L):
    """Argument checks of fam_batch2d_create run before any device call."""
    ci = ctypes.c_int * 2
    nx, ny, k = ci(16, 20), ci(12, 8), ci(5, 4)
    h = ctypes.c_void_p()
    L.fam_batch2d_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_void_p]
    args = lambda **kw: [ctypes.byref(h), kw.get("n", 2), kw.get("nx", nx), kw.get("ny", ny), kw.get("k", k),
                         0.0, 1.0, 0.0, kw.get("y1", 1.0), kw.get("eq", 2), kw.get("bc", 0), 1.4,
                         kw.get("prec", 64), None]
    assert L.fam_batch2d_create(*args(ny=None)) == 1
    assert L.fam_batch2d_create(*args(n=0)) == 1
    assert L.fam_batch2d_create(*args(k=ci(5, 7))) == 1
    assert L.fam_batch2d_create(*args(ny=ci(12, 3))) == 1
    assert L.fam_batch2d_create(*args(y1=0.0)) == 1
    assert L.fam_batch2d_create(*args(bc=2)) == 1
    assert L.fam_batch2d_create(*args(eq=0)) == 7  # FAM_E_UNSUPPORTED: the 2D batch is for 2D Euler
    assert not h.value


def test_null_handle_calls_are_rejected(L):
    assert L.fam_batch_tile(None, None, None) == 1
    assert L.fam_step(None, 0.3) == 1
    assert L.fam_sync(None) == 1
    assert L.fam_set_option(None, b"oe_type", 2.0) == 1
    assert L.fam_last_error(None) == b"null handle"
    L.fam_destroy(None)
    assert L.fam_status_string(4) == b"FAM_E_NONPHYSICAL"


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(fam, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fam, "_lib", None)
    with pytest.raises(FileNotFoundError):
        fam.lib()
