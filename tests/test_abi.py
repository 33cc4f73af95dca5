"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ibm.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(ibm_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2402_17337_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "ibm_step" in names and "ibm_create_grid" in names and "ibm_set_body" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2402_17337_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(ImportError):
        pkg.lib()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2402_17337_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cpp", ".cuh")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "ibm_oracle" not in txt, fn
