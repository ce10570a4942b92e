"""CPU oracle for projective TSDF integration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding in ``paper_2410_21149_gb300``) never does, and shares no code with
it.

`oracle.cpp` states the integrator of coVoxSLAM Sec. III-C/III-D in FP64 with
the FP32 band traversal; `mlp.py` states the per-point weight network in FP64.
This module compiles the C++ with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_L = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _L
    with _lock:
        if _L is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, i64, f32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_int
            L.orc_create.restype = vp
            L.orc_create.argtypes = [f32, f32, f32, i32]
            L.orc_destroy.argtypes = [vp]
            L.orc_num_blocks.restype = i64
            L.orc_num_blocks.argtypes = [vp]
            L.orc_traverse.restype = i32
            L.orc_traverse.argtypes = [vp, vp, vp, i32]
            L.orc_point_obs.restype = i32
            L.orc_point_obs.argtypes = [vp, vp, f32, f32, f32, f32, i32, i32, i32, f32, vp, vp, vp,
                                        i32, vp]
            L.orc_integrate.restype = i32
            L.orc_integrate.argtypes = [vp, vp, i64, vp, vp, i32, i32, f32, f32, i32, vp, i32, vp]
            L.orc_extract_colors.argtypes = [vp, vp]
            L.orc_integrate_parallel.restype = i32
            L.orc_integrate_parallel.argtypes = [vp, vp, i64, vp, vp, i32, i32, f32, f32, i32, vp, i32, i32]
            L.orc_extract.argtypes = [vp, vp, vp, vp]
            L.orc_block_set.restype = i64
            L.orc_block_set.argtypes = [vp, vp, vp, i32, f32, f32, f32, f32, vp, vp, vp, i64]
            L.orc_sampled.argtypes = [vp, vp, vp, vp, i32, f32, f32, f32, i32, i32, i32, f32, f32,
                                      vp, vp, i64, vp, vp, vp]
            L.orc_round_half.argtypes = [vp, i64, vp]
            _L = L
    return _L


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class OracleSubmap:
    """One submap: std::map of 8^3 blocks with FP64 D and W per voxel."""

    def __init__(self, voxel_size: float, trunc: float, max_weight: float = 1e4, fp16: bool = False):
        self.vs, self.trunc, self.max_weight, self.fp16 = voxel_size, trunc, max_weight, fp16
        self.h = lib().orc_create(voxel_size, trunc, max_weight, int(fp16))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def integrate(self, points: np.ndarray, T: np.ndarray, point_weights: Optional[np.ndarray] = None,
                  weight_mode: int = 0, dropoff: int = 0, min_range: float = 0.1,
                  max_range: float = 1e9, sensor: int = 0, carve: bool = False,
                  colors: Optional[np.ndarray] = None) -> Dict[str, int]:
        """One frame; returns the frame's counts and status (0 or -4 key range).
        carve: traverse from the sensor origin (free-space carving).  colors:
        per-point RGB [n,3] fused into the voxels with the same weights."""
        pts = _f32(points).reshape(-1, 3)
        Tm = _f32(T).reshape(12)
        pw = None if point_weights is None else _f32(point_weights)
        rgb = None if colors is None else _f32(colors).reshape(-1, 3)
        stats = np.zeros(6, dtype=np.int64)
        rc = lib().orc_integrate(self.h, _p(pts), len(pts), _p(Tm), _p(pw), weight_mode, dropoff,
                                 min_range, max_range, sensor, _p(stats), 1 if carve else 0, _p(rgb))
        keys = ("valid", "obs", "voxels", "blocks", "new_blocks", "key_range")
        out = dict(zip(keys, (int(x) for x in stats)))
        out["status"] = rc
        return out

    def integrate_parallel(self, points: np.ndarray, T: np.ndarray, threads: int,
                           point_weights: Optional[np.ndarray] = None, weight_mode: int = 0, dropoff: int = 0,
                           min_range: float = 0.1, max_range: float = 1e9, sensor: int = 0,
                           carve: bool = False) -> Dict[str, int]:
        """One frame with its sums accumulated by `threads` threads over point
        chunks (chunk maps added in chunk order): integrate() up to FP64
        rounding, for the timed parallel CPU baseline."""
        pts = _f32(points).reshape(-1, 3)
        Tm = _f32(T).reshape(12)
        pw = None if point_weights is None else _f32(point_weights)
        stats = np.zeros(6, dtype=np.int64)
        rc = lib().orc_integrate_parallel(self.h, _p(pts), len(pts), _p(Tm), _p(pw), weight_mode, dropoff,
                                          min_range, max_range, sensor, _p(stats), 1 if carve else 0,
                                          int(threads))
        keys = ("valid", "obs", "voxels", "blocks", "new_blocks", "key_range")
        out = dict(zip(keys, (int(x) for x in stats)))
        out["status"] = rc
        return out

    @property
    def num_blocks(self) -> int:
        return int(lib().orc_num_blocks(self.h))

    def extract_colors(self) -> np.ndarray:
        """Fused colours float64 [nb, 3, 512] in the order of extract()."""
        C = np.zeros((self.num_blocks, 3, 512), dtype=np.float64)
        lib().orc_extract_colors(self.h, _p(C))
        return C

    def extract(self):
        """(keys int32 [nb,3], D float64 [nb,512], W float64 [nb,512]) sorted by key."""
        nb = self.num_blocks
        keys = np.zeros((nb, 3), dtype=np.int32)
        D = np.zeros((nb, 512), dtype=np.float64)
        W = np.zeros((nb, 512), dtype=np.float64)
        lib().orc_extract(self.h, _p(keys), _p(D), _p(W))
        return keys, D, W


def traverse(A, B) -> np.ndarray:
    """Voxels visited by the FP32 traversal of segment A -> B (voxel units)."""
    A, B = _f32(A), _f32(B)
    cap = 4096
    out = np.zeros((cap, 3), dtype=np.int32)
    n = lib().orc_traverse(_p(A), _p(B), _p(out), cap)
    assert n >= 0
    return out[:n].copy()


def point_obs(ps, T, vs, trunc, min_range=0.1, max_range=1e9, weight_mode=0, dropoff=0,
              sensor=0, point_weight=1.0):
    """Observations of one point: (voxels [m,3], d [m], w [m], segment A|B [6]) or None."""
    ps, Tm = _f32(ps), _f32(T).reshape(12)
    cap = 4096
    vox = np.zeros((cap, 3), dtype=np.int32)
    d = np.zeros(cap)
    w = np.zeros(cap)
    seg = np.zeros(6, dtype=np.float32)
    n = lib().orc_point_obs(_p(ps), _p(Tm), vs, trunc, min_range, max_range, weight_mode, dropoff,
                            sensor, point_weight, _p(vox), _p(d), _p(w), cap, _p(seg))
    if n == 0:
        return None
    if n == -2:
        raise OverflowError("key range")
    assert n > 0
    return vox[:n].copy(), d[:n].copy(), w[:n].copy(), seg


def _scan_arrays(scans: Sequence[np.ndarray], poses: Sequence[np.ndarray]):
    pts = [_f32(s).reshape(-1, 3) for s in scans]
    ptrs = (ctypes.c_void_p * len(pts))(*[p.ctypes.data for p in pts])
    counts = np.array([len(p) for p in pts], dtype=np.int64)
    P = np.ascontiguousarray(np.stack([_f32(T).reshape(12) for T in poses]), dtype=np.float32)
    return pts, ptrs, counts, P


def _weight_ptrs(point_weights):
    if point_weights is None:
        return None, None
    pwl = [_f32(w) for w in point_weights]
    return pwl, (ctypes.c_void_p * len(pwl))(*[w.ctypes.data for w in pwl])


def block_set(scans, poses, vs, trunc, min_range=0.1, max_range=1e9, sensors=None,
              point_weights=None) -> np.ndarray:
    """Sorted int32 [nb,3] keys of every block the scans' bands touch (with
    per-point weights, points whose weight is not finite and >= 0 are dropped)."""
    pts, ptrs, counts, P = _scan_arrays(scans, poses)
    sens = np.ascontiguousarray(sensors if sensors is not None else np.zeros(len(pts)), dtype=np.int32)
    pwl, pwp = _weight_ptrs(point_weights)
    n = lib().orc_block_set(ptrs, _p(counts), _p(P), len(pts), vs, trunc, min_range, max_range,
                            _p(sens), pwp, None, 0)
    keys = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib().orc_block_set(ptrs, _p(counts), _p(P), len(pts), vs, trunc, min_range, max_range,
                        _p(sens), pwp, _p(keys), n)
    return keys[:n]


def sampled(scans, poses, vox, vs, trunc, max_weight=1e4, fp16=False, weight_mode=0, dropoff=0,
            min_range=0.1, max_range=1e9, sensors=None, point_weights=None):
    """Final (D, W, n_obs) of sample voxels [ns,3] after integrating scans frame by frame."""
    pts, ptrs, counts, P = _scan_arrays(scans, poses)
    vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
    ns = len(vox)
    D, W = np.zeros(ns), np.zeros(ns)
    nobs = np.zeros(ns, dtype=np.int64)
    sens = np.ascontiguousarray(sensors if sensors is not None else np.zeros(len(pts)), dtype=np.int32)
    pwl, pwp = _weight_ptrs(point_weights)
    lib().orc_sampled(ptrs, _p(counts), _p(P), pwp, len(pts), vs, trunc, max_weight, int(fp16),
                      weight_mode, dropoff, min_range, max_range, _p(sens), _p(vox), ns, _p(D),
                      _p(W), _p(nobs))
    return D, W, nobs


def round_half(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().orc_round_half(_p(x), x.size, _p(out))
    return out
