"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads and exports
every entry point the header declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

from paper_2608_24109_b300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "exmesh.h")).read()
    return sorted(set(re.findall(r"^\s*(?:exm_status|void|const char\*)\s+(exm_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    decl = declared_entry_points()
    assert len(decl) >= 18
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(decl) == sorted(native.EXPORTS)


def test_binding_signatures_cover_exports():
    native.lib()
    for name in native.EXPORTS:
        fn = getattr(native.lib(), name)
        assert fn.argtypes is not None, name


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "libexmesh.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(ImportError):
        native.lib()


def test_no_cpu_fallback_in_product_path():
    pkg = os.path.join(ROOT, "paper_2608_24109_b300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
