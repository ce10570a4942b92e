"""FP64 oracle of the learned per-point integration weight -- TEST
INFRASTRUCTURE ONLY (tests, smoke and the benchmark's CPU leg).

The paper motivates sensor-dependent weighting and notes that ray casting lets
every point carry its own weight (coVoxSLAM Sec. III-C, weighting paragraph);
the learned weight itself is this project's addition.  Definitions written
here, plainly, in FP64:

features (organised scan, sensor frame, P(v, u) the point of row v, col u):
  f1 = r / max_range,             r = |P|
  f2 = theta / (pi/2),            cos theta = |n . P| / (|n| |P|),
                                  n = (P(v,u+1) - P(v,u-1)) x (P(v+1,u) - P(v-1,u));
                                  theta = 0 when a neighbour is missing/invalid
  f3 = ln(var + 1e-8) / 10,       var = population variance of the depths
                                  (z for a pinhole, range for a spherical
                                  sensor) of the valid points of the 5x5 window
                                  (window clipped at the border), 0 if fewer
                                  than 3 are valid
network (BF16 operands, wider accumulation, bf16() = round to nearest even):
  h1 = relu(bf16(W1) bf16(x) + b1)          W1 [32,3]
  h2 = relu(bf16(W2) bf16(h1) + b2)         W2 [32,32]
  o  = W3 . bf16(h2) + b3                   W3 [32]
  w  = softplus(o)
loss per point with target e2 (mean squared residual of its observations
against the noise-free TSDF): L = w e2 - ln w (Gaussian negative log
likelihood of precision w; optimum w = 1 / e2), averaged over valid points.
Backward mirrors the forward with the same BF16 roundings of the GEMM
operands (dh2 and dh1 rounded before they enter a GEMM).
"""
from __future__ import annotations

import math
from typing import Dict

import numpy as np

H1 = 32
H2 = 32
N_IN = 3


def bf16(x) -> np.ndarray:
    """Round FP64/FP32 values to bfloat16 (round to nearest, ties to even),
    returned as FP64.  Rounds the FP32 value of x, as a device does."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    out[nan] = np.nan
    return out.reshape(np.shape(x))


def softplus(o):
    o = np.asarray(o, dtype=np.float64)
    return np.where(o > 30.0, o, np.log1p(np.exp(np.minimum(o, 30.0))))


def sigmoid(o):
    o = np.asarray(o, dtype=np.float64)
    return 0.5 * (1.0 + np.tanh(0.5 * o))


def init_params(seed: int = 0) -> Dict[str, np.ndarray]:
    """He-style initialisation; b3 set so the initial weight is ~1."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, math.sqrt(2.0 / N_IN), (H1, N_IN)),
        "b1": np.zeros(H1),
        "W2": rng.normal(0, math.sqrt(2.0 / H1), (H2, H1)),
        "b2": np.zeros(H2),
        "W3": rng.normal(0, math.sqrt(1.0 / H2), H2),
        "b3": np.array([0.5413]),   # softplus(0.5413) = 1
    }


ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(v: np.ndarray) -> Dict[str, np.ndarray]:
    shapes = {"W1": (H1, N_IN), "b1": (H1,), "W2": (H2, H1), "b2": (H2,), "W3": (H2,), "b3": (1,)}
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def forward(p, x, rounding: bool = True):
    """x [N,3] -> (w [N], cache).  rounding=False gives the plain FP64 network
    (used by the finite-difference pins)."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    xb = r(x)
    a1 = xb @ r(p["W1"]).T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    h1b = r(h1)
    a2 = h1b @ r(p["W2"]).T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    h2b = r(h2)
    o = h2b @ p["W3"] + p["b3"][0]
    w = softplus(o)
    return w, {"xb": xb, "a1": a1, "h1b": h1b, "a2": a2, "h2b": h2b, "o": o, "rounding": rounding}


def loss(w, e2, mask):
    m = mask.astype(bool)
    n = max(int(m.sum()), 1)
    return float(np.sum((w * e2 - np.log(w))[m]) / n)


def backward(p, cache, w, e2, mask):
    """Gradients of loss() with respect to every parameter."""
    r = bf16 if cache["rounding"] else (lambda a: np.asarray(a, dtype=np.float64))
    m = mask.astype(np.float64)
    n = max(int(m.sum()), 1)
    dw = (e2 - 1.0 / w) * m / n
    do = dw * sigmoid(cache["o"])
    g = {"W3": cache["h2b"].T @ do, "b3": np.array([do.sum()])}
    dh2 = np.outer(do, p["W3"]) * (cache["a2"] > 0)
    g["b2"] = dh2.sum(axis=0)
    dh2b = r(dh2)
    g["W2"] = dh2b.T @ cache["h1b"]
    dh1 = (dh2b @ r(p["W2"])) * (cache["a1"] > 0)
    g["b1"] = dh1.sum(axis=0)
    dh1b = r(dh1)
    g["W1"] = dh1b.T @ cache["xb"]
    return g


class Adam:
    """Adam (Kingma & Ba) on the flattened parameter vector, FP64."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def features(points: np.ndarray, height: int, width: int, sensor: int, max_range: float) -> np.ndarray:
    """[N,3] features of an organised scan (definitions in the module doc)."""
    P = np.asarray(points, dtype=np.float64).reshape(height, width, 3)
    fin = np.isfinite(P).all(axis=2)
    valid = fin & ((P[..., 2] > 0) if sensor == 0 else True)
    r = np.linalg.norm(np.where(valid[..., None], P, 0.0), axis=2)
    depth = P[..., 2] if sensor == 0 else r
    out = np.zeros((height, width, 3))
    for v in range(height):
        for u in range(width):
            if not valid[v, u]:
                continue
            out[v, u, 0] = r[v, u] / max_range
            th = 0.0
            if 0 < u < width - 1 and 0 < v < height - 1 and valid[v, u - 1] and valid[v, u + 1] \
                    and valid[v - 1, u] and valid[v + 1, u]:
                n = np.cross(P[v, u + 1] - P[v, u - 1], P[v + 1, u] - P[v - 1, u])
                nn = np.linalg.norm(n)
                if nn > 0:
                    c = min(abs(n @ P[v, u]) / (nn * r[v, u]), 1.0)
                    th = math.acos(c)
            out[v, u, 1] = th / (math.pi / 2)
            zs = [depth[y, x] for y in range(max(v - 2, 0), min(v + 3, height))
                  for x in range(max(u - 2, 0), min(u + 3, width)) if valid[y, x]]
            var = 0.0
            if len(zs) >= 3:
                mu = sum(zs) / len(zs)
                var = sum((z - mu) ** 2 for z in zs) / len(zs)
            out[v, u, 2] = math.log(var + 1e-8) / 10.0
    return out.reshape(-1, 3)


def targets(points, T, keys, D, W, vs, trunc, min_range=0.1, max_range=1e9, sensor=0):
    """Per-point training target e2 = mean over the point's band voxels whose
    noise-free weight W > 0 of (d - D_clean)^2, and a validity mask (a valid
    point with at least one such voxel).  keys/D/W: the noise-free submap."""
    from . import point_obs
    lut = {}
    for b, k in enumerate(np.asarray(keys)):
        lut[(int(k[0]), int(k[1]), int(k[2]))] = b
    pts = np.asarray(points, dtype=np.float32).reshape(-1, 3)
    e2 = np.zeros(len(pts))
    mask = np.zeros(len(pts), dtype=bool)
    for i, ps in enumerate(pts):
        r = point_obs(ps, T, vs, trunc, min_range, max_range, 0, 0, sensor)
        if r is None:
            continue
        vox, d, _, _ = r
        acc, n = 0.0, 0
        for v, dv in zip(vox, d):
            b = lut.get((int(v[0]) >> 3, int(v[1]) >> 3, int(v[2]) >> 3))
            if b is None:
                continue
            l = (int(v[0]) & 7) + 8 * (int(v[1]) & 7) + 64 * (int(v[2]) & 7)
            if W[b, l] > 0:
                acc += (dv - D[b, l]) ** 2
                n += 1
        if n:
            e2[i] = acc / n
            mask[i] = True
    return e2, mask
