"""Oracle of the submap ESDF and of the backend's submap queries (registration
points, bounds) -- TEST INFRASTRUCTURE ONLY (tests, smoke and the benchmark's
CPU leg).

coVoxSLAM computes a Euclidean signed-distance field from the TSDF blocks
(Sec. III-E, following the Parallel Banding Algorithm); the paper does not
fix the site rule, the sign or a cap, so this oracle states one reading:

  site voxels  S = { allocated voxels with W > w_min and |D| <= site_band }
  ESDF(v)      = vs * min over s in S of || i(v) - i(s) ||_2   for every
                 voxel v of every allocated block (i = integer voxel index,
                 distances between voxel centres), capped at max_dist;
                 max_dist when S is empty.

Unsigned: the distance to the nearest surface voxel.  Everything before the
final scale is exact integer arithmetic (squared distances in voxel units).

Two implementations: `esdf_bruteforce` (every voxel against every site,
small inputs) and `esdf` (the exact separable transform on the dense grid
spanning the allocated blocks: per axis, the lower envelope of the parabolas
(q - p)^2 + f(p), intersections compared as exact integer fractions).
"""
from __future__ import annotations

import numpy as np

INF = np.int64(1) << 60


def _voxel_index(keys: np.ndarray) -> np.ndarray:
    """[nb,512,3] integer voxel indices of the blocks' voxels (local index
    lx + 8 ly + 64 lz)."""
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], 1)
    return keys.astype(np.int64)[:, None, :] * 8 + loc[None, :, :]


def sites(D: np.ndarray, W: np.ndarray, site_band: float, w_min: float) -> np.ndarray:
    """[nb,512] bool site mask."""
    return (W > w_min) & (np.abs(D) <= site_band)


def esdf_bruteforce(keys, D, W, vs, site_band, w_min, max_dist) -> np.ndarray:
    """[nb,512] float64 by direct minimisation (small inputs only)."""
    idx = _voxel_index(np.asarray(keys)).reshape(-1, 3)
    s = idx[sites(np.asarray(D), np.asarray(W), site_band, w_min).reshape(-1)]
    out = np.full(idx.shape[0], float(max_dist))
    if len(s):
        for a in range(0, idx.shape[0], 4096):
            d2 = ((idx[a:a + 4096, None, :] - s[None, :, :]) ** 2).sum(-1).min(1)
            out[a:a + 4096] = np.minimum(np.sqrt(d2.astype(np.float64)) * vs, max_dist)
    return out.reshape(len(keys), 512)


def edt1d(f: np.ndarray) -> np.ndarray:
    """min over p of (q - p)^2 + f[p] for every q (f int64, INF = no site)."""
    n = len(f)
    out = np.full(n, INF, dtype=np.int64)
    v = []              # parabola vertices of the envelope
    zn, zd = [], []     # left boundary of each parabola's interval, as num / den (den > 0)
    for q in range(n):
        if f[q] >= INF:
            continue
        fq = int(f[q]) + q * q
        while v:
            p = v[-1]
            num, den = fq - (int(f[p]) + p * p), 2 * (q - p)   # intersection s = num / den
            if zd[-1] == 0 or num * zd[-1] > zn[-1] * den:      # s > z[k] (z[0] = -inf)
                v.append(q)
                zn.append(num)
                zd.append(den)
                break
            v.pop()
            zn.pop()
            zd.pop()
        else:
            v.append(q)
            zn.append(0)
            zd.append(0)   # -inf
    if not v:
        return out
    k = 0
    for q in range(n):
        while k + 1 < len(v) and zn[k + 1] <= q * zd[k + 1]:   # z[k+1] <= q
            k += 1
        out[q] = (q - v[k]) ** 2 + int(f[v[k]])
    return out


def esdf(keys, D, W, vs, site_band, w_min, max_dist) -> np.ndarray:
    """[nb,512] float64 through the separable exact transform."""
    keys = np.asarray(keys)
    if len(keys) == 0:
        return np.zeros((0, 512))
    idx = _voxel_index(keys)
    lo = idx.reshape(-1, 3).min(0)
    dims = idx.reshape(-1, 3).max(0) - lo + 1
    grid = np.full(tuple(dims), INF, dtype=np.int64)
    m = sites(np.asarray(D), np.asarray(W), site_band, w_min)
    si = idx[m] - lo
    grid[si[:, 0], si[:, 1], si[:, 2]] = 0
    for ax in range(3):
        g = np.moveaxis(grid, ax, -1)
        flat = g.reshape(-1, g.shape[-1])
        res = np.empty_like(flat)
        for r in range(flat.shape[0]):
            res[r] = edt1d(flat[r])
        grid = np.moveaxis(res.reshape(g.shape), -1, ax)
    rel = (idx - lo).reshape(-1, 3)
    d2 = grid[rel[:, 0], rel[:, 1], rel[:, 2]].astype(np.float64)
    out = np.where(d2 >= float(INF), float(max_dist), np.minimum(np.sqrt(d2) * vs, max_dist))
    return out.reshape(len(keys), 512)


def registration_points(keys, D, W, vs, w_min, d_band) -> np.ndarray:
    """Centres (submap frame, metres, ((i + 1/2) * vs) rounded to FP32) of the
    allocated voxels with W >= w_min, W > 0 and |D| <= d_band -- the points the
    backend's registration takes from a submap by their weights (Sec. III-F;
    the selection rule is this project's reading).  Rows sorted."""
    keys = np.asarray(keys)
    D = np.asarray(D, np.float32)
    W = np.asarray(W, np.float32)
    take = (W >= np.float32(w_min)) & (W > 0) & (np.abs(D) <= np.float32(d_band))
    idx = _voxel_index(keys)[take].astype(np.float32)
    c = (idx + np.float32(0.5)) * np.float32(vs)
    return c[np.lexsort((c[:, 2], c[:, 1], c[:, 0]))] if len(c) else c.reshape(0, 3)


def submap_bounds(keys, vs) -> np.ndarray:
    """Block-corner box of the allocated blocks: lo xyz, hi xyz (FP32 metres)."""
    keys = np.asarray(keys).astype(np.float32)
    bs = np.float32(8) * np.float32(vs)
    return np.concatenate([keys.min(0) * bs, (keys.max(0) + 1) * bs]).astype(np.float32)


def submap_overlap(bounds_i, T_i, bounds_j, T_j):
    """Intersection of two posed submaps' boxes (Sec. III-F, the backend's AABB
    overlap test), FP64: each block-corner box (submap frame) carried to the
    world frame by its pose (3x4 world <- submap) as the axis-aligned box of
    its 8 transformed corners, the two boxes intersected.  Returns (volume,
    lo_hi [6]); volume 0 when disjoint or when a box is empty (lo > hi)."""
    def world(b, T):
        b = np.asarray(b, np.float64)
        T = np.asarray(T, np.float64).reshape(3, 4)
        corners = np.array([[b[3] if c & 1 else b[0], b[4] if c & 2 else b[1], b[5] if c & 4 else b[2]]
                            for c in range(8)])
        w = corners @ T[:, :3].T + T[:, 3]
        return w.min(0), w.max(0)

    bi, bj = np.asarray(bounds_i, np.float64), np.asarray(bounds_j, np.float64)
    li, hi_ = world(bi, T_i)
    lj, hj = world(bj, T_j)
    lo, hi = np.maximum(li, lj), np.minimum(hi_, hj)
    empty = (bi[:3] > bi[3:]).any() or (bj[:3] > bj[3:]).any()
    vol = 0.0 if empty else float(np.prod(np.maximum(hi - lo, 0.0)))
    return vol, np.concatenate([lo, hi])

