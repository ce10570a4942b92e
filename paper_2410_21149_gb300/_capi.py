"""ctypes binding of libcovox.so (include/covox.h): argument marshalling only.

Every function keeps the C name and forwards device pointers of torch tensors
and the raw CUDA stream handle; all integration work runs in the library's
CUDA kernels.  There is no CPU path: if the library is missing or CUDA is not
available the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcovox.so")

CVX_OK, CVX_ERR_INVALID_ARG, CVX_ERR_OOM, CVX_ERR_CAPACITY = 0, -1, -2, -3
CVX_ERR_KEY_RANGE, CVX_ERR_TIMEOUT, CVX_ERR_CUDA = -4, -5, -6
CVX_STORE_F32, CVX_STORE_F16 = 0, 1
CVX_W_CONST, CVX_W_QUADRATIC, CVX_W_PER_POINT = 0, 1, 2
CVX_DROP_NONE, CVX_DROP_LINEAR, CVX_DROP_QUADRATIC = 0, 1, 2
CVX_SENSOR_PINHOLE, CVX_SENSOR_SPHERICAL = 0, 1
CVX_SUBMAP_PIPELINED = 1
CVX_SUBMAP_FOUR_SETS = 2
CVX_SUBMAP_COLOR = 4
CVX_INTEGRATE_CARVE = 1

STATUS_NAMES = {0: "CVX_OK", -1: "CVX_ERR_INVALID_ARG", -2: "CVX_ERR_OOM", -3: "CVX_ERR_CAPACITY",
                -4: "CVX_ERR_KEY_RANGE", -5: "CVX_ERR_TIMEOUT", -6: "CVX_ERR_CUDA"}


class CovoxError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")
        self.status = status


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class cvx_submap_params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("trunc", ctypes.c_float),
                ("max_weight", ctypes.c_float), ("storage", ctypes.c_int32),
                ("max_blocks", ctypes.c_int64), ("hash_slots", ctypes.c_int64),
                ("flags", ctypes.c_int64), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class cvx_integrate_params(ctypes.Structure):
    _fields_ = [("weight_mode", ctypes.c_int32), ("dropoff", ctypes.c_int32),
                ("min_range", ctypes.c_float), ("max_range", ctypes.c_float),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("sensor", ctypes.c_int32), ("pts_per_cta", ctypes.c_int32),
                ("local_blocks", ctypes.c_int32), ("flags", ctypes.c_int32)]


class cvx_counters(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int64), ("frames", ctypes.c_int64),
                ("valid_points", ctypes.c_int64), ("observations", ctypes.c_int64),
                ("voxels_merged", ctypes.c_int64), ("blocks_touched", ctypes.c_int64)]


class cvx_scan_desc(ctypes.Structure):
    _fields_ = [("submap", ctypes.c_int32), ("pad", ctypes.c_int32), ("points_xyz", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("T_sub_sensor", ctypes.c_float * 12),
                ("point_weights", ctypes.c_void_p), ("params", cvx_integrate_params),
                ("colors_rgb", ctypes.c_void_p)]


class cvx_submap_view(ctypes.Structure):
    _fields_ = [("hash_keys", ctypes.c_void_p), ("hash_vals", ctypes.c_void_p),
                ("hash_slots", ctypes.c_int64), ("block_keys", ctypes.c_void_p),
                ("dist", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("state", ctypes.c_void_p),
                ("max_blocks", ctypes.c_int64), ("voxel_size", ctypes.c_float),
                ("trunc", ctypes.c_float), ("max_weight", ctypes.c_float)]


CVX_NOALLOC_MAX_BLOCKS = 4096
CVX_SUBMAP_STATE_BYTES = 128

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/covox.h
_vp, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
SIGNATURES = {
    "cvx_version": (ctypes.c_char_p, []),
    "cvx_create_submap": (_i32, [ctypes.POINTER(cvx_submap_params), ctypes.POINTER(_vp)]),
    "cvx_integrate_scan": (_i32, [_vp, _vp, _i64, _vp, _vp, ctypes.POINTER(cvx_integrate_params), _vp]),
    "cvx_integrate_scan_color": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, ctypes.POINTER(cvx_integrate_params), _vp]),
    "cvx_extract_blocks": (_i32, [_vp, _i64, _vp, _vp, _vp, ctypes.POINTER(_i64), _vp]),
    "cvx_extract_colors": (_i32, [_vp, _i64, _vp, ctypes.POINTER(_i64), _vp]),
    "cvx_reset_submap": (_i32, [_vp, _vp]),
    "cvx_reset_submaps": (_i32, [ctypes.POINTER(_vp), _i32, _vp]),
    "cvx_submap_status": (_i32, [_vp]),
    "cvx_flush_submap": (_i32, [_vp, _vp]),
    "cvx_registration_points": (_i32, [_vp, ctypes.c_float, ctypes.c_float, _i64, _vp, _vp, _vp]),
    "cvx_submap_bounds": (_i32, [_vp, _vp, _vp]),
    "cvx_submap_overlaps": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "cvx_block_hash_create": (_i32, [_i64, _i64, _vp]),
    "cvx_block_hash_insert": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "cvx_block_hash_find": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "cvx_block_hash_info": (_i32, [_vp, _vp, _vp, _i64]),
    "cvx_block_hash_destroy": (None, [_vp]),
    "cvx_compute_esdf": (_i32, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
    "cvx_submap_counters": (_i32, [_vp, ctypes.POINTER(cvx_counters)]),
    "cvx_destroy": (None, [_vp]),
    "cvx_integrate_scan_noalloc": (_i32, [ctypes.POINTER(cvx_submap_view), _vp, _i64, _vp, _vp,
                                          ctypes.POINTER(cvx_integrate_params), _vp]),
    "cvx_batch_create": (_i32, [_i32, _i32, ctypes.POINTER(_vp)]),
    "cvx_integrate_batch": (_i32, [_vp, ctypes.POINTER(_vp), _i32, ctypes.POINTER(cvx_scan_desc), _i32, _vp]),
    "cvx_batch_error": (_i32, [_vp]),
    "cvx_batch_destroy": (None, [_vp]),
    "cvx_batch_timing": (_i32, [_vp, _i32]),
    "cvx_batch_wave_limit": (_i32, [_vp, _i32]),
    "cvx_batch_merge_parts": (_i32, [_vp, _i32]),
    "cvx_batch_submap_group": (_i32, [_vp, _i32]),
    "cvx_batch_test_missing_cta": (_i32, [_vp, _i32, _i64]),
    "cvx_batch_phase_times": (_i32, [_vp, _vp, _i32]),
    "cvx_point_features": (_i32, [_vp, _i32, _i32, _i32, ctypes.c_float, _vp, _vp]),
    "cvx_weight_model_create": (_i32, [_vp, ctypes.POINTER(_vp)]),
    "cvx_weight_model_params": (_i32, [_vp, _vp, _vp, _vp]),
    "cvx_weight_model_infer": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "cvx_weight_model_point_weights": (_i32, [_vp, _vp, _i32, _i32, _i32, ctypes.c_float, _vp, _vp]),
    "cvx_weight_model_point_weights_frames": (_i32, [_vp, _vp, _i32, _i32, _i32, _i32, ctypes.c_float, _vp, _vp]),
    "cvx_weight_model_train_step": (_i32, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, _vp]),
    "cvx_weight_model_last": (_i32, [_vp, _vp, _vp, _vp]),
    "cvx_weight_model_destroy": (None, [_vp]),
    "cvx_training_targets": (_i32, [_vp, _vp, _i64, _vp, ctypes.POINTER(cvx_integrate_params), _vp, _vp, _vp]),
    "cvx_normalise_targets": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "cvx_profile_start": (_i32, [_i64]),
    "cvx_profile_stop": (_i32, []),
    "cvx_profile_read": (_i32, [_i32, _vp, _vp, _vp]),
    "cvx_launch_count": (_i64, []),
}


def lib():
    """Load libcovox.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_2410_21149_gb300._build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != CVX_OK:
        raise CovoxError(status, what)


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t, dtype_name: str, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != dtype_name or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous {dtype_name} tensor")
    return t.data_ptr()


# ------------------------------------------------------------ entry points
def cvx_version() -> str:
    return lib().cvx_version().decode()


def cvx_create_submap(params: cvx_submap_params) -> int:
    h = ctypes.c_void_p()
    check(lib().cvx_create_submap(ctypes.byref(params), ctypes.byref(h)), "cvx_create_submap")
    return h.value


def cvx_integrate_scan(handle: int, points, T_sub_sensor, point_weights, params: cvx_integrate_params,
                       stream=None) -> None:
    n = int(points.shape[0])
    pp = _dev_ptr(points, "torch.float32", "points") if n else None
    pw = None if point_weights is None else _dev_ptr(point_weights, "torch.float32", "point_weights")
    T = np.ascontiguousarray(T_sub_sensor, dtype=np.float32).reshape(12)
    check(lib().cvx_integrate_scan(handle, pp, n, T.ctypes.data_as(ctypes.c_void_p), pw,
                                   ctypes.byref(params), _stream_handle(stream)), "cvx_integrate_scan")


def cvx_integrate_scan_color(handle: int, points, T_sub_sensor, point_weights, colors,
                             params: cvx_integrate_params, stream=None) -> None:
    n = int(points.shape[0])
    pp = _dev_ptr(points, "torch.float32", "points") if n else None
    pw = None if point_weights is None else _dev_ptr(point_weights, "torch.float32", "point_weights")
    pc = _dev_ptr(colors, "torch.float32", "colors") if n else None
    T = np.ascontiguousarray(T_sub_sensor, dtype=np.float32).reshape(12)
    check(lib().cvx_integrate_scan_color(handle, pp, n, T.ctypes.data_as(ctypes.c_void_p), pw, pc,
                                         ctypes.byref(params), _stream_handle(stream)), "cvx_integrate_scan_color")


def cvx_extract_colors(handle: int, capacity: int, rgb, stream=None) -> int:
    n = ctypes.c_int64(0)
    check(lib().cvx_extract_colors(handle, capacity, None if rgb is None else rgb.data_ptr(), ctypes.byref(n),
                                   _stream_handle(stream)), "cvx_extract_colors")
    return n.value


def cvx_batch_create(max_submaps: int, max_scans: int) -> int:
    h = ctypes.c_void_p()
    check(lib().cvx_batch_create(max_submaps, max_scans, ctypes.byref(h)), "cvx_batch_create")
    return h.value


def cvx_integrate_batch(batch: int, maps, scans, stream=None) -> None:
    """maps: submap handles; scans: list of (submap index, points tensor,
    T (12 floats), point_weights tensor or None, cvx_integrate_params[,
    colours tensor [n,3] for colour submaps])."""
    arr_maps = (ctypes.c_void_p * len(maps))(*maps)
    descs = (cvx_scan_desc * max(len(scans), 1))()
    for k, sc in enumerate(scans):
        mi, pts, T, pw, prm = sc[:5]
        col = sc[5] if len(sc) > 5 else None
        n = int(pts.shape[0])
        descs[k].colors_rgb = None if col is None or n == 0 else _dev_ptr(col, "torch.float32", "colors")
        descs[k].submap = int(mi)
        descs[k].points_xyz = _dev_ptr(pts, "torch.float32", "points") if n else None
        descs[k].n = n
        descs[k].T_sub_sensor[:] = [float(x) for x in np.asarray(T, dtype=np.float32).reshape(12)]
        descs[k].point_weights = None if pw is None else _dev_ptr(pw, "torch.float32", "point_weights")
        descs[k].params = prm
    check(lib().cvx_integrate_batch(batch, arr_maps, len(maps), descs, len(scans), _stream_handle(stream)),
          "cvx_integrate_batch")


def cvx_batch_error(batch: int) -> int:
    return int(lib().cvx_batch_error(batch))


def cvx_batch_wave_limit(batch: int, max_scans_per_wave: int) -> None:
    check(lib().cvx_batch_wave_limit(batch, int(max_scans_per_wave)), "cvx_batch_wave_limit")


def cvx_batch_submap_group(batch: int, group: int) -> None:
    check(lib().cvx_batch_submap_group(batch, int(group)), "cvx_batch_submap_group")


def cvx_batch_merge_parts(batch: int, parts: int) -> None:
    check(lib().cvx_batch_merge_parts(batch, int(parts)), "cvx_batch_merge_parts")


def cvx_batch_test_missing_cta(batch: int, missing_cta: int, barrier_polls: int = 0) -> None:
    check(lib().cvx_batch_test_missing_cta(batch, int(missing_cta), int(barrier_polls)),
          "cvx_batch_test_missing_cta")


def cvx_batch_timing(batch: int, enable: bool) -> None:
    check(lib().cvx_batch_timing(batch, int(enable)), "cvx_batch_timing")


def cvx_batch_phase_times(batch: int, max_scans: int = 1 << 16) -> np.ndarray:
    """[scans, 3] milliseconds from the launch start to each scan's tiles done
    and merge done (third column 0), scans in queue order."""
    out = np.zeros(3 * max_scans, np.float64)
    n = lib().cvx_batch_phase_times(batch, out.ctypes.data_as(ctypes.c_void_p), max_scans)
    if n < 0:
        raise CovoxError(n, "cvx_batch_phase_times")
    return out[:3 * n].reshape(n, 3)


def cvx_batch_destroy(batch: int) -> None:
    if batch:
        lib().cvx_batch_destroy(batch)


def cvx_integrate_scan_noalloc(view: cvx_submap_view, points, T_sub_sensor, point_weights,
                               params: cvx_integrate_params, stream=None) -> int:
    """Returns the status (no exception) so callers can see CVX_ERR_CAPACITY."""
    n = int(points.shape[0])
    pp = _dev_ptr(points, "torch.float32", "points") if n else None
    pw = None if point_weights is None else _dev_ptr(point_weights, "torch.float32", "point_weights")
    T = np.ascontiguousarray(T_sub_sensor, dtype=np.float32).reshape(12)
    return int(lib().cvx_integrate_scan_noalloc(ctypes.byref(view), pp, n, T.ctypes.data_as(ctypes.c_void_p),
                                                pw, ctypes.byref(params), _stream_handle(stream)))


def cvx_extract_blocks(handle: int, capacity: int, keys, dist, weight, stream=None) -> int:
    n = ctypes.c_int64(0)
    ptr = (lambda t: None if t is None else t.data_ptr())
    check(lib().cvx_extract_blocks(handle, capacity, ptr(keys), ptr(dist), ptr(weight), ctypes.byref(n),
                                   _stream_handle(stream)), "cvx_extract_blocks")
    return n.value


def cvx_reset_submap(handle: int, stream=None) -> None:
    check(lib().cvx_reset_submap(handle, _stream_handle(stream)), "cvx_reset_submap")


def cvx_reset_submaps(handles, stream=None) -> None:
    arr = (_vp * max(len(handles), 1))(*handles)
    check(lib().cvx_reset_submaps(arr, len(handles), _stream_handle(stream)), "cvx_reset_submaps")


def cvx_compute_esdf(handle: int, site_band: float, w_min: float, max_dist: float, out, sq_dist=None,
                     stream=None) -> None:
    """out: float32 CUDA tensor [n_blocks, 512]; sq_dist: int32 CUDA tensor of the
    same shape or None."""
    o = _dev_ptr(out, "torch.float32", "out")
    q = _dev_ptr(sq_dist, "torch.int32", "sq_dist") if sq_dist is not None else None
    check(lib().cvx_compute_esdf(handle, float(site_band), float(w_min), float(max_dist), o, q,
                                 _stream_handle(stream)), "cvx_compute_esdf")


def cvx_registration_points(handle: int, w_min: float, d_band: float, xyz=None, stream=None) -> int:
    """Writes into xyz (float32 CUDA tensor [capacity,3]) if given; returns the
    number of qualifying voxels (synchronous)."""
    n = ctypes.c_int64(0)
    cap = int(xyz.shape[0]) if xyz is not None else 0
    ptr = _dev_ptr(xyz, "torch.float32", "xyz") if cap else None
    check(lib().cvx_registration_points(handle, float(w_min), float(d_band), cap, ptr, ctypes.byref(n),
                                        _stream_handle(stream)), "cvx_registration_points")
    return int(n.value)


def cvx_submap_bounds(handle: int, stream=None) -> np.ndarray:
    out = np.zeros(6, np.float32)
    check(lib().cvx_submap_bounds(handle, out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)),
          "cvx_submap_bounds")
    return out


def cvx_submap_overlaps(bounds, poses, with_boxes: bool = False, stream=None):
    """bounds: device float32 [n,6]; poses: device float32 [n,12] (world <-
    submap).  Returns (volume [n,n], boxes [n,n,6] or None) device tensors."""
    import torch
    n = int(bounds.shape[0])
    vol = torch.empty((n, n), dtype=torch.float32, device=bounds.device)
    boxes = torch.empty((n, n, 6), dtype=torch.float32, device=bounds.device) if with_boxes else None
    check(lib().cvx_submap_overlaps(n, _dev_ptr(bounds, "torch.float32", "bounds"),
                                    _dev_ptr(poses, "torch.float32", "poses"), vol.data_ptr(),
                                    None if boxes is None else boxes.data_ptr(), _stream_handle(stream)),
          "cvx_submap_overlaps")
    return vol, boxes


def cvx_block_hash_create(slots: int, max_blocks: int) -> int:
    h = ctypes.c_void_p()
    check(lib().cvx_block_hash_create(int(slots), int(max_blocks), ctypes.byref(h)), "cvx_block_hash_create")
    return h.value


def cvx_block_hash_insert(handle: int, coords, pool, stream=None) -> None:
    """coords: int32 CUDA tensor [n,3]; pool: int32 CUDA tensor [n] (output)."""
    n = int(coords.shape[0])
    check(lib().cvx_block_hash_insert(handle, _dev_ptr(coords, "torch.int32", "coords") if n else None, n,
                                      _dev_ptr(pool, "torch.int32", "pool") if n else None,
                                      _stream_handle(stream)), "cvx_block_hash_insert")


def cvx_block_hash_find(handle: int, coords, pool, stream=None) -> None:
    n = int(coords.shape[0])
    check(lib().cvx_block_hash_find(handle, _dev_ptr(coords, "torch.int32", "coords") if n else None, n,
                                    _dev_ptr(pool, "torch.int32", "pool") if n else None,
                                    _stream_handle(stream)), "cvx_block_hash_find")


def cvx_block_hash_info(handle: int, with_keys: bool = False):
    """(status, n_blocks, block keys int32 [n,3] numpy array or None); synchronous."""
    nb = ctypes.c_int64(0)
    st = int(lib().cvx_block_hash_info(handle, ctypes.byref(nb), None, 0))
    keys = None
    if with_keys and nb.value > 0:
        keys = np.zeros((nb.value, 3), np.int32)
        st = int(lib().cvx_block_hash_info(handle, ctypes.byref(nb), keys.ctypes.data_as(ctypes.c_void_p),
                                           nb.value))
    return st, int(nb.value), keys


def cvx_block_hash_destroy(handle: int) -> None:
    lib().cvx_block_hash_destroy(handle)


def cvx_flush_submap(handle: int, stream=None) -> None:
    check(lib().cvx_flush_submap(handle, _stream_handle(stream)), "cvx_flush_submap")


def cvx_submap_status(handle: int) -> int:
    return int(lib().cvx_submap_status(handle))


def cvx_submap_counters(handle: int) -> dict:
    c = cvx_counters()
    check(lib().cvx_submap_counters(handle, ctypes.byref(c)), "cvx_submap_counters")
    return {f: int(getattr(c, f)) for f, _ in cvx_counters._fields_}


def cvx_destroy(handle: int) -> None:
    if handle:
        lib().cvx_destroy(handle)


def cvx_profile_start(max_launches: int = 1 << 20) -> None:
    check(lib().cvx_profile_start(max_launches), "cvx_profile_start")


def cvx_profile_stop() -> None:
    check(lib().cvx_profile_stop(), "cvx_profile_stop")


def cvx_profile_read() -> dict:
    """{kernel name: (total ms, timed launches)} since the last read (synchronises)."""
    k = 32   # at least the library's number of kernel kinds
    names = ctypes.create_string_buffer(32 * k)
    tot = np.zeros(k, np.float64)
    cnt = np.zeros(k, np.int64)
    n = lib().cvx_profile_read(k, names, tot.ctypes.data_as(ctypes.c_void_p),
                               cnt.ctypes.data_as(ctypes.c_void_p))
    raw = names.raw
    out = {}
    for q in range(n):
        name = raw[32 * q:32 * q + 32].split(b"\0")[0].decode()
        out[name] = (float(tot[q]), int(cnt[q]))
    return out


def cvx_launch_count() -> int:
    return int(lib().cvx_launch_count())


CVX_MLP_PARAMS = 1217


def cvx_point_features(points, height: int, width: int, sensor: int, max_range: float, out, stream=None):
    check(lib().cvx_point_features(_dev_ptr(points, "torch.float32", "points"), height, width, sensor,
                                   float(max_range), _dev_ptr(out, "torch.float32", "features"),
                                   _stream_handle(stream)), "cvx_point_features")


def cvx_weight_model_create(init_params: np.ndarray) -> int:
    p = np.ascontiguousarray(init_params, dtype=np.float32).reshape(CVX_MLP_PARAMS)
    h = ctypes.c_void_p()
    check(lib().cvx_weight_model_create(p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
          "cvx_weight_model_create")
    return h.value


def cvx_weight_model_params(model: int, set_params=None, get=False, stream=None):
    sp = None
    if set_params is not None:
        sp = np.ascontiguousarray(set_params, dtype=np.float32).reshape(CVX_MLP_PARAMS)
    out = np.zeros(CVX_MLP_PARAMS, np.float32) if get else None
    check(lib().cvx_weight_model_params(model, None if sp is None else sp.ctypes.data_as(ctypes.c_void_p),
                                        None if out is None else out.ctypes.data_as(ctypes.c_void_p),
                                        _stream_handle(stream)), "cvx_weight_model_params")
    if sp is not None and not get:
        import torch
        torch.cuda.current_stream().synchronize()   # the host copy is read asynchronously
    return out


def cvx_weight_model_infer(model: int, features, weights_out, stream=None):
    n = int(features.shape[0])
    check(lib().cvx_weight_model_infer(model, _dev_ptr(features, "torch.float32", "features"), n,
                                       _dev_ptr(weights_out, "torch.float32", "weights"), _stream_handle(stream)),
          "cvx_weight_model_infer")


def cvx_weight_model_point_weights(model: int, points, height: int, width: int, sensor: int, max_range: float,
                                   weights_out, stream=None):
    check(lib().cvx_weight_model_point_weights(model, _dev_ptr(points, "torch.float32", "points"), int(height),
                                               int(width), int(sensor), float(max_range),
                                               _dev_ptr(weights_out, "torch.float32", "weights"),
                                               _stream_handle(stream)), "cvx_weight_model_point_weights")


def cvx_weight_model_point_weights_frames(model: int, points, n_frames: int, height: int, width: int, sensor: int,
                                          max_range: float, weights_out, stream=None):
    """points: CUDA float32 [n_frames, height*width, 3] (or flat); weights_out [n_frames, height*width]."""
    if points.numel() != 3 * n_frames * height * width or weights_out.numel() != n_frames * height * width:
        raise ValueError("points / weights do not hold n_frames scans of height x width")
    check(lib().cvx_weight_model_point_weights_frames(model, _dev_ptr(points, "torch.float32", "points"),
                                                      int(n_frames), int(height), int(width), int(sensor),
                                                      float(max_range),
                                                      _dev_ptr(weights_out, "torch.float32", "weights"),
                                                      _stream_handle(stream)),
          "cvx_weight_model_point_weights_frames")


def cvx_weight_model_train_step(model: int, features, e2, mask, lr: float, stream=None):
    n = int(features.shape[0])
    check(lib().cvx_weight_model_train_step(model, _dev_ptr(features, "torch.float32", "features"),
                                            _dev_ptr(e2, "torch.float32", "e2"), _dev_ptr(mask, "torch.float32", "mask"),
                                            n, float(lr), _stream_handle(stream)), "cvx_weight_model_train_step")


def cvx_weight_model_last(model: int, stream=None):
    g = np.zeros(CVX_MLP_PARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    check(lib().cvx_weight_model_last(model, g.ctypes.data_as(ctypes.c_void_p), loss.ctypes.data_as(ctypes.c_void_p),
                                      _stream_handle(stream)), "cvx_weight_model_last")
    return g, float(loss[0])


def cvx_weight_model_destroy(model: int) -> None:
    if model:
        lib().cvx_weight_model_destroy(model)


def cvx_training_targets(clean_handle: int, points, T_sub_sensor, params, e2_out, mask_out, stream=None):
    n = int(points.shape[0])
    T = np.ascontiguousarray(T_sub_sensor, dtype=np.float32).reshape(12)
    check(lib().cvx_training_targets(clean_handle, _dev_ptr(points, "torch.float32", "points") if n else None, n,
                                     T.ctypes.data_as(ctypes.c_void_p), ctypes.byref(params),
                                     _dev_ptr(e2_out, "torch.float32", "e2"),
                                     _dev_ptr(mask_out, "torch.float32", "mask"), _stream_handle(stream)),
          "cvx_training_targets")


def cvx_normalise_targets(e2, mask, stream=None) -> float:
    """Divide e2 (device float32 [n]) in place by its mean over mask; returns the mean."""
    n = int(e2.shape[0])
    out = ctypes.c_float(0.0)
    check(lib().cvx_normalise_targets(_dev_ptr(e2, "torch.float32", "e2"), _dev_ptr(mask, "torch.float32", "mask"),
                                      n, ctypes.byref(out), _stream_handle(stream)), "cvx_normalise_targets")
    return float(out.value)
