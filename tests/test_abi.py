"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (no device calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(mr_[a-z_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1905_08717_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mr_create", "mr_adapt", "mr_step", "mr_read", "mr_destroy", "mr_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_config_is_rejected_without_device_work(lib):
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.burgers_1d(L=6)
    bad = p.replace(rk_order=4)
    cfg = pkg.make_config(bad)
    h = ctypes.c_void_p()
    lib.mr_create.argtypes = [ctypes.POINTER(pkg.mr_config), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    r = lib.mr_create(ctypes.byref(cfg), q.ctypes.data, None, ctypes.byref(h))
    assert r == 1 and not h.value
    lib.mr_last_error.restype = ctypes.c_char_p
    assert lib.mr_last_error(None) == b"null handle"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1905_08717_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.library()
