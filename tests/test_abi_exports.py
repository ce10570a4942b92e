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


def test_noalloc_rejects_misaligned_views_on_the_host():
    """The allocation-free entry point checks the caller's view before any
    CUDA call: a pointer off its alignment (D and W 16 bytes, hash keys and
    state 8, hash values and block keys 4) gives CVX_ERR_INVALID_ARG, and an
    oversized view CVX_ERR_CAPACITY.  The pointers are never dereferenced."""
    import numpy as np
    from paper_2410_21149_gb300 import _build, _capi
    _build.build()
    L = _capi.lib()
    T = np.eye(3, 4, dtype=np.float32).reshape(12)
    prm = _capi.cvx_integrate_params(0, 0, 0.1, 1e9, 0, 0, 0, 0, 0, 0)

    def view(**off):
        base = {"hash_keys": 0x10000, "hash_vals": 0x20000, "block_keys": 0x30000, "dist": 0x40000,
                "weight": 0x50000, "state": 0x60000}
        v = _capi.cvx_submap_view()
        for k, a in base.items():
            setattr(v, k, a + off.get(k, 0))
        v.hash_slots, v.max_blocks = 1024, 64
        v.voxel_size, v.trunc, v.max_weight = 0.1, 0.3, 1e4
        return v

    def call(v):
        return L.cvx_integrate_scan_noalloc(ctypes.byref(v), None, 0, T.ctypes.data_as(ctypes.c_void_p), None,
                                            ctypes.byref(prm), None)

    for field, off in (("dist", 4), ("weight", 8), ("hash_keys", 4), ("state", 4), ("hash_vals", 2),
                       ("block_keys", 1)):
        assert call(view(**{field: off})) == _capi.CVX_ERR_INVALID_ARG, field
    big = view()
    big.max_blocks = _capi.CVX_NOALLOC_MAX_BLOCKS + 1
    assert call(big) == _capi.CVX_ERR_CAPACITY
