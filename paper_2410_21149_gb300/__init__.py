"""GB300-native projective TSDF integration into block-hashed voxel submaps.

The hot path of coVoxSLAM's submap mapping (Sec. III-B/C/D): hand-written
sm_103a CUDA kernels behind the C ABI of include/covox.h (libcovox.so).  This
package is the thin Python binding: `_capi` mirrors the C entry points by
name; `Submap` owns one submap whose device memory comes from PyTorch's
caching allocator through the library's allocator hooks.  PyTorch provides
device memory and streams only.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _capi
from ._capi import (CVX_DROP_LINEAR, CVX_DROP_NONE, CVX_DROP_QUADRATIC, CVX_SENSOR_PINHOLE,
                    CVX_SENSOR_SPHERICAL, CVX_STORE_F16, CVX_STORE_F32, CVX_W_CONST,
                    CVX_W_PER_POINT, CVX_W_QUADRATIC, CovoxError, cvx_integrate_params,
                    cvx_submap_params)

__all__ = ["Submap", "CovoxError", "integrate_params", "_capi"]


def _torch_allocator():
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream if stream else 0)
        except Exception:  # noqa: BLE001 -- reported as CVX_ERR_OOM by the library
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return _capi.ALLOC_FN(alloc), _capi.FREE_FN(free)


def integrate_params(weight_mode=CVX_W_CONST, dropoff=CVX_DROP_NONE, min_range=0.1,
                     max_range=1e9, sensor=CVX_SENSOR_PINHOLE, height=0, width=0,
                     pts_per_cta=0, local_blocks=0, carve=False) -> cvx_integrate_params:
    return cvx_integrate_params(int(weight_mode), int(dropoff), float(min_range), float(max_range),
                                int(height), int(width), int(sensor), int(pts_per_cta),
                                int(local_blocks), _capi.CVX_INTEGRATE_CARVE if carve else 0)


class Submap:
    """One block-hashed TSDF submap on the current CUDA device."""

    def __init__(self, voxel_size: float, trunc: float, max_weight: float = 1e4,
                 storage: int = CVX_STORE_F32, max_blocks: int = 1 << 16,
                 hash_slots: Optional[int] = None,
                 use_torch_allocator: bool = True, stream=None, pipelined: bool = False, sets: int = 0,
                 color: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Submap needs a CUDA device; there is no CPU path")
        if hash_slots is None:
            hash_slots = 1 << max(1, int(np.ceil(np.log2(2 * max_blocks))))
        self._fns = _torch_allocator() if use_torch_allocator else (_capi.ALLOC_FN(), _capi.FREE_FN())
        flags = (_capi.CVX_SUBMAP_FOUR_SETS if sets == 4 else
                 (_capi.CVX_SUBMAP_PIPELINED if (pipelined or sets == 2) else 0))
        flags |= _capi.CVX_SUBMAP_COLOR if color else 0
        p = cvx_submap_params(float(voxel_size), float(trunc), float(max_weight), int(storage),
                              int(max_blocks), int(hash_slots), int(flags),
                              self._fns[0], self._fns[1], None, _capi._stream_handle(stream))
        self.voxel_size, self.trunc, self.max_weight, self.storage = voxel_size, trunc, max_weight, storage
        self.max_blocks, self.hash_slots, self.color = max_blocks, hash_slots, color
        self.handle = _capi.cvx_create_submap(p)

    def close(self):
        if getattr(self, "handle", None):
            _capi.cvx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def integrate(self, points, T_sub_sensor, params: cvx_integrate_params, point_weights=None,
                  stream=None, colors=None) -> None:
        """colors: CUDA float32 [n,3] per-point colours (required by colour submaps)."""
        if colors is None:
            _capi.cvx_integrate_scan(self.handle, points, T_sub_sensor, point_weights, params, stream)
        else:
            _capi.cvx_integrate_scan_color(self.handle, points, T_sub_sensor, point_weights, colors, params,
                                           stream)

    def reset(self, stream=None) -> None:
        _capi.cvx_reset_submap(self.handle, stream)

    def esdf(self, site_band: Optional[float] = None, w_min: float = 0.0, max_dist: float = 2.0,
             exact_sq: bool = False, stream=None):
        """Distance field of the allocated voxels ([nb, 512] float32 CUDA tensor in
        extract() block order; with exact_sq also the int32 squared distances in
        voxel units).  site_band defaults to the voxel size."""
        import torch
        nb = self.num_blocks(stream)
        out = torch.empty((max(nb, 1), 512), dtype=torch.float32, device="cuda")
        sq = torch.empty((max(nb, 1), 512), dtype=torch.int32, device="cuda") if exact_sq else None
        band = self.voxel_size if site_band is None else site_band
        _capi.cvx_compute_esdf(self.handle, band, w_min, max_dist, out, sq, stream)
        return (out[:nb], sq[:nb]) if exact_sq else out[:nb]

    def flush(self, stream=None) -> None:
        """Merge the scan a pipelined submap left pending (no-op otherwise)."""
        _capi.cvx_flush_submap(self.handle, stream)

    def status(self) -> int:
        return _capi.cvx_submap_status(self.handle)

    def counters(self) -> dict:
        return _capi.cvx_submap_counters(self.handle)

    def num_blocks(self, stream=None) -> int:
        return _capi.cvx_extract_blocks(self.handle, 0, None, None, None, stream)

    def extract(self, stream=None):
        """(keys int32 [nb,3], D [nb,512], W [nb,512]) as CUDA tensors in allocation
        order; float32 storage gives D in metres, float16 gives D / trunc."""
        import torch
        nb = self.num_blocks(stream)
        dt = torch.float32 if self.storage == CVX_STORE_F32 else torch.float16
        keys = torch.empty((max(nb, 1), 3), dtype=torch.int32, device="cuda")
        D = torch.empty((max(nb, 1), 512), dtype=dt, device="cuda")
        W = torch.empty((max(nb, 1), 512), dtype=dt, device="cuda")
        n = _capi.cvx_extract_blocks(self.handle, nb, keys, D, W, stream)
        return keys[:n], D[:n], W[:n]

    def extract_colors(self, stream=None):
        """Fused colours [nb, 3, 512] float32 CUDA tensor, blocks in extract() order."""
        import torch
        nb = _capi.cvx_extract_colors(self.handle, 0, None, stream)
        C = torch.empty((max(nb, 1), 3, 512), dtype=torch.float32, device="cuda")
        n = _capi.cvx_extract_colors(self.handle, nb, C, stream)
        return C[:n]
