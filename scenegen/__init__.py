"""Seeded synthetic scenes, trajectories and range scans.

Input generation only: nothing here computes any part of the integration
method.  Both the CPU oracle (``oracle/``) and the CUDA path consume exactly
the float32 scans and poses produced here, and the analytic scene distance
(`Scene.sdf`) is the ground truth for the SDF RMSE metric.

The scenes stand in for the paper's datasets (Sec. IV: ARCHE MAV LiDAR
flights, Replica/Redwood RGB-D), which are not available; their shapes follow
the five workload configurations listed in ``WORKLOADS``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_SO = os.path.join(_HERE, "libscenegen.so")
_lock = threading.Lock()
_lib_handle = None

SG_ROOM, SG_BOX, SG_SPHERE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile libscenegen.so next to its source (gcc, OpenMP, no arch flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, dp, fp, i64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64
            L.sg_scene_create.restype = vp
            L.sg_scene_create.argtypes = [vp, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double]
            L.sg_scene_destroy.argtypes = [vp]
            L.sg_sdf.argtypes = [vp, dp, i64, ctypes.c_double, dp]
            L.sg_render_pinhole.restype = i64
            L.sg_render_pinhole.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, fp]
            L.sg_render_lidar.restype = i64
            L.sg_render_lidar.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_uint64, ctypes.c_uint64, fp]
            L.sg_trace_rays.argtypes = [vp, dp, dp, i64, ctypes.c_double, dp]
            L.sg_terrain_height.restype = ctypes.c_double
            L.sg_terrain_height.argtypes = [vp, ctypes.c_double, ctypes.c_double]
            _lib_handle = L
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Scene:
    """A procedural scene: primitives (rooms, boxes, spheres) plus optional terrain."""

    def __init__(self, prims: list, terrain: Optional[dict] = None, grid_res: float = 2.0):
        self.prims = prims
        self.types = np.array([p[0] for p in prims], dtype=np.int32)
        self.params = np.zeros((max(len(prims), 1), 6), dtype=np.float64)
        for k, p in enumerate(prims):
            self.params[k, :len(p[1])] = p[1]
        self.terrain = terrain
        L = _lib()
        if terrain is not None:
            h = np.ascontiguousarray(terrain["h"], dtype=np.float64)
            self._h = h
            self.handle = L.sg_scene_create(_ptr(self.types), _ptr(self.params), len(prims),
                                            _ptr(h), h.shape[1], h.shape[0], terrain["x0"],
                                            terrain["y0"], terrain["res"], grid_res)
        else:
            self.handle = L.sg_scene_create(_ptr(self.types), _ptr(self.params), len(prims),
                                            None, 0, 0, 0.0, 0.0, 1.0, grid_res)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib().sg_scene_destroy(h)
            self.handle = None

    def sdf(self, pts: np.ndarray, cap: float) -> np.ndarray:
        """Analytic signed distance (positive in free space), clamped to [-cap, cap]."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.empty(len(p), dtype=np.float64)
        _lib().sg_sdf(self.handle, _ptr(p), len(p), float(cap), _ptr(out))
        return out

    def trace(self, o: np.ndarray, d: np.ndarray, tmax: float) -> np.ndarray:
        o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        out = np.empty(len(o), dtype=np.float64)
        _lib().sg_trace_rays(self.handle, _ptr(o), _ptr(d), len(o), float(tmax), _ptr(out))
        return out

    def terrain_height(self, x: float, y: float) -> float:
        return float(_lib().sg_terrain_height(self.handle, float(x), float(y)))


# ---------------------------------------------------------------- sensors
@dataclasses.dataclass
class Pinhole:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    max_depth: float
    noise_kind: int = 0      # 0 none, 1 along-ray sigma, 2 axial k*z^2
    noise_k: float = 0.0
    dropout: float = 0.0
    sensor: int = 0          # integration sensor model: 0 = pinhole (z = optical axis)

    def render(self, scene: Scene, T_ws: np.ndarray, seed: int, scan_id: int) -> np.ndarray:
        out = np.empty((self.height * self.width, 3), dtype=np.float32)
        T = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(12)
        _lib().sg_render_pinhole(scene.handle, _ptr(T), self.width, self.height, self.fx, self.fy,
                                 self.cx, self.cy, self.max_depth, self.noise_kind, self.noise_k,
                                 self.dropout, seed, scan_id, _ptr(out))
        return out


@dataclasses.dataclass
class Lidar:
    rows: int = 64
    cols: int = 1024
    el_min: float = -math.radians(16.6)
    el_max: float = math.radians(16.6)
    max_range: float = 50.0
    sigma: float = 0.02
    sensor: int = 1          # integration sensor model: 1 = spherical (z = range)

    @property
    def height(self):
        return self.rows

    @property
    def width(self):
        return self.cols

    def render(self, scene: Scene, T_ws: np.ndarray, seed: int, scan_id: int) -> np.ndarray:
        out = np.empty((self.rows * self.cols, 3), dtype=np.float32)
        T = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(12)
        _lib().sg_render_lidar(scene.handle, _ptr(T), self.rows, self.cols, self.el_min,
                               self.el_max, self.max_range, self.sigma, seed, scan_id, _ptr(out))
        return out


# ------------------------------------------------------------------ poses
def pose_from(R: np.ndarray, t) -> np.ndarray:
    T = np.zeros((3, 4), dtype=np.float64)
    T[:, :3] = R
    T[:, 3] = t
    return T


def look_frame(forward, down_hint=(0.0, 0.0, -1.0)) -> np.ndarray:
    """Camera rotation (columns x right, y down, z forward) for a pinhole sensor."""
    z = np.asarray(forward, dtype=np.float64)
    z = z / np.linalg.norm(z)
    y = np.asarray(down_hint, dtype=np.float64)
    y = y - z * (y @ z)
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    return np.stack([x, y, z], axis=1)


def lidar_frame(forward) -> np.ndarray:
    """LiDAR rotation (columns x forward, y left, z up), horizontal forward axis."""
    f = np.array([forward[0], forward[1], 0.0], dtype=np.float64)
    f /= np.linalg.norm(f)
    z = np.array([0.0, 0.0, 1.0])
    y = np.cross(z, f)
    return np.stack([f, y, z], axis=1)


# ----------------------------------------------------------------- scenes
def room_scene(seed: int = 1):
    """10 x 10 x 3 m room with 5 spheres (r ~ U[0.3, 0.8]) and 3 boxes."""
    rng = np.random.default_rng(seed)
    prims = [(SG_ROOM, [0, 0, 0, 10, 10, 3])]
    c = np.array([5.0, 5.0])
    for _ in range(5):
        r = rng.uniform(0.3, 0.8)
        a = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(3.9, 4.4) - r * 0.5
        p = c + rad * np.array([math.cos(a), math.sin(a)])
        prims.append((SG_SPHERE, [p[0], p[1], rng.uniform(r, 3.0 - r), r]))
    for _ in range(3):
        s = rng.uniform(0.3, 1.5, size=3)
        a = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(4.0, 4.6) - 0.5 * max(s[0], s[1])
        p = c + rad * np.array([math.cos(a), math.sin(a)])
        lo = [p[0] - s[0] / 2, p[1] - s[1] / 2, 0.0]
        prims.append((SG_BOX, lo + [lo[0] + s[0], lo[1] + s[1], s[2]]))
    return Scene(prims, grid_res=2.0)


def multiroom_scene(seed: int = 2):
    """30 x 30 x 5 m building: 3 x 3 rooms, 0.2 m walls with door gaps, furniture."""
    rng = np.random.default_rng(seed)
    prims = [(SG_ROOM, [0, 0, 0, 30, 30, 5])]
    th, door_w, door_h = 0.2, 1.2, 2.2
    for wpos in (10.0, 20.0):
        for axis in (0, 1):
            for seg in range(3):
                a0, a1 = seg * 10.0, seg * 10.0 + 10.0
                dc = rng.uniform(a0 + 2.0, a1 - 2.0)
                parts = [(a0, dc - door_w / 2, 0.0, 5.0), (dc + door_w / 2, a1, 0.0, 5.0),
                         (dc - door_w / 2, dc + door_w / 2, door_h, 5.0)]
                for (s0, s1, z0, z1) in parts:
                    if axis == 0:   # wall at x = wpos spanning y
                        prims.append((SG_BOX, [wpos - th / 2, s0, z0, wpos + th / 2, s1, z1]))
                    else:           # wall at y = wpos spanning x
                        prims.append((SG_BOX, [s0, wpos - th / 2, z0, s1, wpos + th / 2, z1]))
    for ri in range(3):
        for rj in range(3):
            x0, y0 = ri * 10.0, rj * 10.0
            for _ in range(3):
                s = rng.uniform(0.4, 1.6, size=3)
                px, py = rng.uniform(x0 + 1.0, x0 + 9.0 - s[0]), rng.uniform(y0 + 1.0, y0 + 9.0 - s[1])
                prims.append((SG_BOX, [px, py, 0.0, px + s[0], py + s[1], s[2]]))
            for _ in range(2):
                r = rng.uniform(0.3, 0.7)
                prims.append((SG_SPHERE, [rng.uniform(x0 + 1.5, x0 + 8.5), rng.uniform(y0 + 1.5, y0 + 8.5),
                                          rng.uniform(r, 2.5), r]))
    return Scene(prims, grid_res=2.0)


def _terrain_heights(seed: int, x0: float, y0: float, res: float, nx: int, ny: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    xs = x0 + res * np.arange(nx)
    ys = y0 + res * np.arange(ny)
    X, Y = np.meshgrid(xs, ys)
    h = np.zeros_like(X)
    for amp, fr in ((2.0, 0.02), (1.0, 0.05), (0.4, 0.13), (0.15, 0.4)):
        for _ in range(2):
            a = rng.uniform(0, 2 * math.pi)
            ph = rng.uniform(0, 2 * math.pi, size=2)
            h += amp * np.sin(fr * (X * math.cos(a) + Y * math.sin(a)) + ph[0]) \
                * np.cos(fr * (-X * math.sin(a) + Y * math.cos(a)) + ph[1])
    return h


def outdoor_scene(seed: int = 3, n_boxes: int = 2000, path_len: float = 400.0):
    """Terrain heightfield, rubble of random boxes and one building shell crossed by
    a closed ~path_len m loop (the MAV flight path).  Returns (scene, path fn)."""
    rng = np.random.default_rng(seed)
    ax, by = 75.0 * path_len / 400.0, 50.0 * path_len / 400.0
    ext = ax + 60.0
    res = 0.5
    nx = int(2 * ext / res) + 1
    ny = int(2 * (by + 60.0) / res) + 1
    terrain = {"x0": -ext, "y0": -(by + 60.0), "res": res,
               "h": _terrain_heights(seed, -ext, -(by + 60.0), res, nx, ny)}
    prims = []
    scene0 = Scene([], terrain)     # terrain-only scene for height queries

    def path_xy(s):                  # s in [0,1): ellipse loop
        a = 2 * math.pi * s
        return ax * math.cos(a), by * math.sin(a)

    ts = np.linspace(0, 1, 4000, endpoint=False)
    pxy = np.array([path_xy(t) for t in ts])
    # building shell straddling the path at s = 0.25 (top of the ellipse)
    bx, byc = path_xy(0.25)
    bw, bd, bh, wt = 20.0, 12.0, 6.0, 0.3
    z0 = scene0.terrain_height(bx, byc) - 1.0
    lo = np.array([bx - bw / 2, byc - bd / 2, z0])
    hi = np.array([bx + bw / 2, byc + bd / 2, z0 + bh])
    door = 4.0
    # east/west walls (x = const) cut by the path, which runs along x near the top
    for xw in (lo[0], hi[0] - wt):
        prims.append((SG_BOX, [xw, lo[1], z0, xw + wt, byc - door / 2, hi[2]]))
        prims.append((SG_BOX, [xw, byc + door / 2, z0, xw + wt, hi[1], hi[2]]))
        prims.append((SG_BOX, [xw, byc - door / 2, z0 + 5.5, xw + wt, byc + door / 2, hi[2]]))
    prims.append((SG_BOX, [lo[0], lo[1], z0, hi[0], lo[1] + wt, hi[2]]))
    prims.append((SG_BOX, [lo[0], hi[1] - wt, z0, hi[0], hi[1], hi[2]]))
    prims.append((SG_BOX, [lo[0], lo[1], hi[2] - wt, hi[0], hi[1], hi[2]]))
    # rubble: boxes scattered near the path, none within 2.5 m of it
    placed = 0
    tries = 0
    while placed < n_boxes and tries < 50 * n_boxes:
        tries += 1
        s = rng.uniform(0, 1)
        cx, cy = path_xy(s)
        off = rng.uniform(-25.0, 25.0, size=2)
        x, y = cx + off[0], cy + off[1]
        size = rng.uniform(0.2, 2.0, size=3)
        dmin = np.min(np.hypot(pxy[:, 0] - x, pxy[:, 1] - y)) - 0.75 * max(size[0], size[1])
        if dmin < 2.5:
            continue
        if lo[0] - 1 < x < hi[0] + 1 and lo[1] - 1 < y < hi[1] + 1:
            continue
        zb = scene0.terrain_height(x, y) - 0.2
        prims.append((SG_BOX, [x - size[0] / 2, y - size[1] / 2, zb,
                               x + size[0] / 2, y + size[1] / 2, zb + size[2]]))
        placed += 1
    scene = Scene(prims, terrain, grid_res=2.0)
    scene.path_xy = path_xy
    scene.building_floor = z0
    return scene


# ------------------------------------------------------------ trajectories
def circle_trajectory(n: int, centre=(5.0, 5.0), radius: float = 3.0, height: float = 1.5):
    poses = []
    for k in range(n):
        a = 2 * math.pi * k / n
        p = [centre[0] + radius * math.cos(a), centre[1] + radius * math.sin(a), height]
        fwd = [math.cos(a), math.sin(a), -0.1]
        poses.append(pose_from(look_frame(fwd), p))
    return poses


def random_walk_trajectory(scene: Scene, n: int, seed: int, start=(5.0, 5.0, 1.5),
                           step: float = 0.1, max_turn_deg: float = 5.0, clearance: float = 0.6):
    rng = np.random.default_rng(seed)
    pos = np.array(start, dtype=np.float64)
    yaw = rng.uniform(0, 2 * math.pi)
    poses = []
    for k in range(n):
        pitch = math.radians(8.0) * math.sin(0.05 * k)
        fwd = [math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)]
        poses.append(pose_from(look_frame(fwd), pos.copy()))
        yaw += math.radians(rng.uniform(-max_turn_deg, max_turn_deg))
        cand = pos + step * np.array([math.cos(yaw), math.sin(yaw), 0.0])
        ahead = pos + 1.0 * np.array([math.cos(yaw), math.sin(yaw), 0.0])
        if scene.sdf(np.stack([cand, ahead]), 5.0).min() < clearance:
            yaw += math.radians(max_turn_deg)     # turn in place, do not move
        else:
            pos = cand
    return poses


def loop_trajectory(scene: Scene, n: int, spacing: float = 0.2, altitude: float = 3.0):
    """n LiDAR poses spaced ~spacing m along the scene's closed loop, at a fixed
    altitude above the terrain (and the building floor inside the building)."""
    ts = np.linspace(0, 1, 20001)
    pts = np.array([scene.path_xy(t) for t in ts])
    seg = np.hypot(np.diff(pts[:, 0]), np.diff(pts[:, 1]))
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    poses = []
    for k in range(n):
        s = (k * spacing) % cum[-1]
        i = min(int(np.searchsorted(cum, s)), len(ts) - 2)
        x, y = pts[i]
        fx, fy = pts[i + 1] - pts[i]
        z = max(scene.terrain_height(x, y), scene.building_floor + 1.0) + altitude \
            + 0.5 * math.sin(0.03 * s)
        poses.append(pose_from(lidar_frame([fx, fy]), [x, y, z]))
    return poses


# ---------------------------------------------------------------- workloads
@dataclasses.dataclass
class Scan:
    points: np.ndarray        # float32 [N, 3], sensor frame, NaN for no return
    T_sub_sensor: np.ndarray  # float32 [12], 3x4 row-major submap <- sensor
    sensor: int               # 0 pinhole, 1 spherical LiDAR
    height: int
    width: int


@dataclasses.dataclass
class SubmapWork:
    scans: List[Scan]
    T_world_sub: np.ndarray   # float64 [3, 4]
    voxel_size: float
    trunc: float
    scene: Optional["Scene"] = None   # scene the submap's scans see (None: the workload's)


@dataclasses.dataclass
class Workload:
    name: str
    submaps: List[SubmapWork]
    max_weight: float
    weight_mode: int          # 0 constant, 1 quadratic 1/z^2, 2 per point
    dropoff: int              # 0 none, 1 linear, 2 quadratic
    min_range: float
    max_range: float
    scene: Scene
    storage: int = 0          # 0 float32, 1 float16

    @property
    def n_points(self) -> int:
        return sum(s.points.shape[0] for sm in self.submaps for s in sm.scans)

    @property
    def n_scans(self) -> int:
        return sum(len(sm.scans) for sm in self.submaps)


def _to_sub(T_ws: np.ndarray, anchor) -> np.ndarray:
    T = T_ws.copy()
    T[:, 3] = T[:, 3] - np.asarray(anchor, dtype=np.float64)
    return np.ascontiguousarray(T.reshape(12), dtype=np.float32)


def make_c1(seed: int = 1, n_frames: int = 10) -> Workload:
    """Room, 10 pinhole frames 160x120 on a circle, sigma = 0.01 m along the ray."""
    scene = room_scene(seed)
    cam = Pinhole(160, 120, 131.25, 131.25, 79.5, 59.5, max_depth=20.0, noise_kind=1, noise_k=0.01)
    scans = [Scan(cam.render(scene, T, seed, k), _to_sub(T, (0, 0, 0)), 0, 120, 160)
             for k, T in enumerate(circle_trajectory(n_frames))]
    sm = SubmapWork(scans, pose_from(np.eye(3), [0, 0, 0]), 0.10, 0.30)
    return Workload("room-160x120x10", [sm], 1e4, 0, 0, 0.1, 20.0, scene)


def make_c2(seed: int = 2, n_frames: int = 200, width: int = 640, height: int = 480,
            storage: int = 0, dropoff: int = 1, noise: bool = True) -> Workload:
    """Multi-room building, pinhole 640x480 on a random walk; axial sigma 0.0012 z^2,
    2% dropout, max depth 10 m; quadratic weight with behind-surface drop-off."""
    scene = multiroom_scene(seed)
    f = 525.0 * width / 640.0
    cam = Pinhole(width, height, f, f, (width - 1) / 2.0, (height - 1) / 2.0, max_depth=10.0,
                  noise_kind=2 if noise else 0, noise_k=0.0012, dropout=0.02 if noise else 0.0)
    traj = random_walk_trajectory(scene, n_frames, seed)
    scans = [Scan(cam.render(scene, T, seed, k), _to_sub(T, (0, 0, 0)), 0, height, width)
             for k, T in enumerate(traj)]
    sm = SubmapWork(scans, pose_from(np.eye(3), [0, 0, 0]), 0.05, 0.15)
    return Workload(f"multiroom-{width}x{height}x{n_frames}", [sm], 1e4, 1, dropoff, 0.1, 10.0,
                    scene, storage)


def make_c3(seed: int = 3, n_scans: int = 2000, scans_per_submap: int = 50, rows: int = 64,
            cols: int = 1024, n_boxes: int = 2000, first_scan: int = 0, scan_stride: int = 1) -> Workload:
    """LiDAR MAV flight: 64x1024 spherical scans 0.2 m apart along a 400 m loop
    through terrain, rubble and a building; a new submap every scans_per_submap
    scans, each submap frame anchored at its first scan's position."""
    scene = outdoor_scene(seed, n_boxes)
    lid = Lidar(rows, cols)
    traj = loop_trajectory(scene, first_scan + n_scans * scan_stride)
    submaps = []
    idx = list(range(first_scan, first_scan + n_scans * scan_stride, scan_stride))
    for s0 in range(0, len(idx), scans_per_submap):
        chunk = idx[s0:s0 + scans_per_submap]
        anchor = traj[chunk[0]][:, 3].copy()
        scans = [Scan(lid.render(scene, traj[k], seed, k), _to_sub(traj[k], anchor), 1, rows, cols)
                 for k in chunk]
        submaps.append(SubmapWork(scans, pose_from(np.eye(3), anchor), 0.20, 0.80))
    return Workload(f"lidar-{rows}x{cols}x{n_scans}", submaps, 1e4, 0, 0, 0.1, 50.0, scene)


def make_c4(seed: int = 4, n_submaps: int = 32, max_scans: int = 16, depth_wh=(640, 480),
            lidar_rc=(64, 1024)) -> Workload:
    """32 submaps of uneven load: each gets 1-16 scans mixing pinhole frames of the
    building and LiDAR scans of the outdoor scene; voxel size per submap in
    {0.05, 0.10, 0.20} m, trunc 3 vs (4 vs for 0.20 m); FP16 storage."""
    rng = np.random.default_rng(seed)
    indoor = multiroom_scene(seed)
    outdoor = outdoor_scene(seed + 1, n_boxes=2000)
    W, H = depth_wh
    f = 525.0 * W / 640.0
    cam = Pinhole(W, H, f, f, (W - 1) / 2.0, (H - 1) / 2.0, max_depth=10.0, noise_kind=2,
                  noise_k=0.0012, dropout=0.02)
    lid = Lidar(*lidar_rc)
    traj_in = random_walk_trajectory(indoor, 400, seed)
    traj_out = loop_trajectory(outdoor, 2000)
    submaps = []
    for m in range(n_submaps):
        n = int(rng.integers(1, max_scans + 1))
        vs = float(rng.choice([0.05, 0.10, 0.20]))
        tr = 4 * vs if vs == 0.20 else 3 * vs
        outdoor_map = bool(rng.integers(0, 2))
        scans = []
        if outdoor_map:
            k0 = int(rng.integers(0, 2000 - 4 * n))
            anchor = traj_out[k0][:, 3].copy()
            for j in range(n):
                k = k0 + 4 * j
                if j % 3 == 2:   # mixed: a pinhole frame looking along the path
                    T = traj_out[k].copy()
                    T[:, :3] = look_frame(T[:, 0], (0, 0, -1))
                    scans.append(Scan(cam.render(outdoor, T, seed, 100000 + m * 64 + j),
                                      _to_sub(T, anchor), 0, H, W))
                else:
                    scans.append(Scan(lid.render(outdoor, traj_out[k], seed, m * 64 + j),
                                      _to_sub(traj_out[k], anchor), 1, lid.rows, lid.cols))
        else:
            k0 = int(rng.integers(0, 400 - 2 * n))
            anchor = traj_in[k0][:, 3].copy()
            for j in range(n):
                k = k0 + 2 * j
                if j % 4 == 3:   # mixed: a LiDAR scan from the camera position
                    T = pose_from(lidar_frame(traj_in[k][:, 2]), traj_in[k][:, 3])
                    scans.append(Scan(lid.render(indoor, T, seed, 200000 + m * 64 + j),
                                      _to_sub(T, anchor), 1, lid.rows, lid.cols))
                else:
                    scans.append(Scan(cam.render(indoor, traj_in[k], seed, 300000 + m * 64 + j),
                                      _to_sub(traj_in[k], anchor), 0, H, W))
        submaps.append(SubmapWork(scans, pose_from(np.eye(3), anchor), vs, tr,
                                  outdoor if outdoor_map else indoor))
    wl = Workload(f"batched-{n_submaps}maps", submaps, 1e4, 0, 0, 0.1, 50.0, indoor, storage=1)
    wl.scenes = {"indoor": indoor, "outdoor": outdoor}
    return wl


WORKLOADS = {
    "c1": make_c1,
    "c2": make_c2,
    "c3": make_c3,
    "c4": make_c4,
}


def point_colors(scan: Scan, seed: int = 0, period: float = 1.5) -> np.ndarray:
    """float32 [N, 3] colours in [0, 1] of a scan's points: a seeded procedural
    albedo of the point's submap-frame position (one sinusoid per channel,
    direction and phase drawn from `seed`, spatial period `period` metres), so
    scans that see the same surface agree up to their range noise.  Points
    without a return get colour 0."""
    rng = np.random.default_rng(10_000 + seed)
    dirs = rng.normal(size=(3, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    phase = rng.uniform(0, 2 * np.pi, 3)
    T = np.asarray(scan.T_sub_sensor, np.float64).reshape(3, 4)
    p = scan.points.astype(np.float64) @ T[:, :3].T + T[:, 3]
    c = 0.5 + 0.5 * np.sin(p @ dirs.T * (2 * np.pi / period) + phase)
    c[~np.isfinite(c).all(axis=1)] = 0.0
    return np.ascontiguousarray(c, dtype=np.float32)
