"""The C ABI library loads and exports every symbol include/ccg.h declares,
and refuses to compute without a GPU (no CPU fallback).  No GPU needed."""
import ctypes
import os
import re

import pytest

from paper_1208_4869_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ccg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("ccg_create", "ccg_destroy", "ccg_op_dense", "ccg_matvec", "ccg_dot", "ccg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_no_cpu_fallback_without_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    L = ctypes.CDLL(libpath)
    L.ccg_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    L.ccg_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    st = L.ccg_create(ctypes.byref(h), None)
    assert st == -3 and not h.value
    assert b"device" in L.ccg_last_error()


def test_binding_raises_when_library_missing(monkeypatch, tmp_path):
    from paper_1208_4869_gb300 import ccg
    monkeypatch.setattr(ccg, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ccg, "_lib", None)
    with pytest.raises(ImportError):
        ccg.lib()


def test_callback_operator_rejects_bad_arguments_without_gpu(libpath):
    """ccg_op_callback validates its arguments before touching a device."""
    L = ctypes.CDLL(libpath)
    fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p)
    L.ccg_op_callback.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, fn, fn, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    op = ctypes.c_void_p(1)
    good = fn(lambda ctx, n, x, y, s: 0)
    assert L.ccg_op_callback(None, 1, 8, good, fn(), None, 0, ctypes.byref(op)) == -1   # no handle
    assert not op.value


def test_server_estimate_without_gpu():
    """The serving admission's byte estimate is host arithmetic: dense
    requests hold both matrices (24 n^2 bytes at least); dipole requests also
    their cached operators (three FFT grids and the field-tensor octant per
    precision), so a larger lattice costs more."""
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg
    d = ccg.server_estimate(kind="dense", n=1024, nrhs=1)
    assert d >= 24 * 1024 * 1024
    assert ccg.server_estimate(kind="dense", n=1024, nrhs=8) > d
    small, big = ccg.server_estimate(kind="dipole", L=16), ccg.server_estimate(kind="dipole", L=32)
    assert big > 7 * small
    assert big >= 3 * 8 * 32 ** 3 * 24
