"""Learned per-point integration weight: features, training targets, the
3-32-32-1 network (trained and evaluated by the library's CUDA kernels), and
the gate that keeps it only where it lowers the SDF error.

coVoxSLAM Sec. III-C (weighting paragraph): weights should follow the
sensor's error curve, and ray casting lets each point carry its own weight.
Training pairs come from the plain integrator: noisy scans are compared with
the TSDF fused from the same scans without noise; the network is fitted by
minimising w e2 - ln w (Gaussian negative log likelihood of precision w).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _capi

N_PARAMS = _capi.CVX_MLP_PARAMS
H = 32


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation (W1 [32,3], b1, W2 [32,32], b2, W3, b3); the
    output bias starts where softplus = 1 (the constant weight)."""
    rng = np.random.default_rng(seed)
    p = [rng.normal(0, np.sqrt(2.0 / 3), (H, 3)).ravel(), np.zeros(H),
         rng.normal(0, np.sqrt(2.0 / H), (H, H)).ravel(), np.zeros(H),
         rng.normal(0, np.sqrt(1.0 / H), H), np.array([0.5413])]
    return np.concatenate(p).astype(np.float32)


def features(points, height: int, width: int, sensor: int, max_range: float, stream=None):
    """Device [N,3] features of an organised scan (points: CUDA float32 [N,3])."""
    import torch
    out = torch.empty((height * width, 3), dtype=torch.float32, device=points.device)
    _capi.cvx_point_features(points, height, width, sensor, max_range, out, stream)
    return out


class WeightModel:
    def __init__(self, params: Optional[np.ndarray] = None, seed: int = 0):
        self.handle = _capi.cvx_weight_model_create(init_params(seed) if params is None else params)

    def close(self):
        if getattr(self, "handle", None):
            _capi.cvx_weight_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    @property
    def params(self) -> np.ndarray:
        return _capi.cvx_weight_model_params(self.handle, get=True)

    @params.setter
    def params(self, p: np.ndarray) -> None:
        _capi.cvx_weight_model_params(self.handle, set_params=p)

    def infer(self, feats, stream=None):
        import torch
        w = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
        _capi.cvx_weight_model_infer(self.handle, feats, w, stream)
        return w

    def train_step(self, feats, e2, mask, lr: float, stream=None) -> None:
        _capi.cvx_weight_model_train_step(self.handle, feats, e2, mask, lr, stream)

    def last(self) -> Tuple[np.ndarray, float]:
        return _capi.cvx_weight_model_last(self.handle)


def training_targets(clean_submap, points, T, params, stream=None):
    """(e2, mask) device arrays of a noisy scan against a noise-free float32 submap."""
    import torch
    n = points.shape[0]
    e2 = torch.empty(n, dtype=torch.float32, device=points.device)
    mask = torch.empty(n, dtype=torch.float32, device=points.device)
    _capi.cvx_training_targets(clean_submap.handle, points, T, params, e2, mask, stream)
    return e2, mask


def build_training_set(noisy_scans: Sequence, clean_scans: Sequence, voxel_size: float, trunc: float,
                       max_range: float, min_range: float = 0.1, max_blocks: int = 1 << 17):
    """Fuse the noise-free scans with the plain integrator (constant weight),
    then compute each noisy point's features and target.  Scans are objects
    with .points, .T_sub_sensor, .sensor, .height, .width and identical poses.
    Returns (feats, e2, mask) with e2 in metres^2 (see normalise_targets)."""
    import torch
    from . import Submap, integrate_params
    clean = Submap(voxel_size, trunc, 1e4, 0, max_blocks=max_blocks)
    for sc in clean_scans:
        clean.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor,
                        integrate_params(0, 0, min_range, max_range, sc.sensor, sc.height, sc.width))
    F, E, M = [], [], []
    for sc in noisy_scans:
        pts = torch.from_numpy(sc.points).cuda()
        prm = integrate_params(0, 0, min_range, max_range, sc.sensor, sc.height, sc.width)
        e2, mask = training_targets(clean, pts, sc.T_sub_sensor, prm)
        F.append(features(pts, sc.height, sc.width, sc.sensor, max_range))
        E.append(e2)
        M.append(mask)
    assert clean.status() == 0
    clean.close()
    return torch.cat(F), torch.cat(E), torch.cat(M)


def normalise_targets(e2, mask):
    """Targets divided by their mean over valid points (cvx_normalise_targets,
    in place on the device): the fitted weights are then ~1 for a typical
    point, the scale of the constant weight.  Returns (e2, mean)."""
    e2 = e2.contiguous()
    mean = _capi.cvx_normalise_targets(e2, mask.contiguous())
    return e2, mean


def train(model: WeightModel, feats, e2, mask, steps: int = 400, batch: int = 65536, lr: float = 3e-3,
          seed: int = 0) -> List[float]:
    """Mini-batch Adam on the GPU; returns the loss of every step."""
    import torch
    g = torch.Generator(device=feats.device)
    g.manual_seed(seed)
    n = feats.shape[0]
    losses = []
    for _ in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=feats.device, generator=g)
        model.train_step(feats[idx].contiguous(), e2[idx].contiguous(), mask[idx].contiguous(), lr)
        losses.append(model.last()[1])
    return losses


def learned_point_weights(model: WeightModel, scan_points, height: int, width: int, sensor: int,
                          max_range: float, out=None, stream=None):
    """Per-point weights of one organised scan (device [N]): features and
    network in one fused kernel."""
    import torch
    w = torch.empty(height * width, dtype=torch.float32, device=scan_points.device) if out is None else out
    _capi.cvx_weight_model_point_weights(model.handle, scan_points, height, width, sensor, max_range, w, stream)
    return w


def learned_point_weights_frames(model: WeightModel, frames_points, height: int, width: int, sensor: int,
                                 max_range: float, out=None, stream=None):
    """Per-point weights of n organised scans of one shape in one launch:
    frames_points CUDA float32 [n, height*width, 3]; returns [n, height*width]."""
    import torch
    n = int(frames_points.shape[0])
    w = torch.empty((n, height * width), dtype=torch.float32, device=frames_points.device) if out is None else out
    _capi.cvx_weight_model_point_weights_frames(model.handle, frames_points, n, height, width, sensor, max_range,
                                                w, stream)
    return w


def gate(rmse_learned: float, rmse_plain: float) -> bool:
    """Keep the learned weight only where it lowers the SDF RMSE against the
    scene (measured by the caller on validation data); otherwise the plain
    constant or quadratic weight stays."""
    return rmse_learned < rmse_plain
