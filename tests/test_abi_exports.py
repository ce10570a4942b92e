"""The C-ABI library loads on the CPU and exports every function that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(cvx_\w+)\s*\(", src):
            if not m.group(1).endswith("_fn"):
                names.add(m.group(1))
    return names


def test_library_exports_all_declared_symbols():
    from paper_2410_21149_gb300 import _build, _capi
    _build.build()
    L = ctypes.CDLL(_capi.LIB_PATH)
    declared = _declared()
    assert {"cvx_create_submap", "cvx_integrate_scan", "cvx_extract_blocks", "cvx_destroy"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    # the binding mirrors every declared entry point by name
    assert declared <= set(_capi.SIGNATURES), declared - set(_capi.SIGNATURES)
    assert _capi.lib().cvx_version().startswith(b"covox")


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2410_21149_gb300 import _capi
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    import pytest
    with pytest.raises(RuntimeError):
        _capi.lib()
