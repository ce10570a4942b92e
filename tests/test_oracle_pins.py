"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties one part of the oracle to a hand-derived value, a closed form,
exact geometry (brute force), an invariant of the weighted-mean update, or a
library routine.  coVoxSLAM Sec. III-C (ray casting, weighting) and
Sec. III-D (count / allocate / commutative per-voxel reduction) define what is
pinned here.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
import scenegen as sg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------- traversal
def test_traversal_hand_cases():
    for case in _load("traversal_hand.json")["cases"]:
        got = orc.traverse(case["A"], case["B"])
        assert got.tolist() == case["voxels"], case["note"]


def _exact_cells(A, B, lo, hi, margin):
    """Cells c in [lo, hi)^3 whose open interior the segment A->B crosses for a
    parameter interval longer than `margin` ("in"), or misses by more than
    `margin` ("out"); everything else is a near tie ("tie").  FP64 slab test."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    d = B - A
    res = {}
    for x in range(lo[0], hi[0]):
        for y in range(lo[1], hi[1]):
            for z in range(lo[2], hi[2]):
                c = np.array([x, y, z], np.float64)
                t0, t1 = 0.0, 1.0
                gap = math.inf
                for k in range(3):
                    if d[k] == 0.0:
                        s = min(A[k] - c[k], c[k] + 1 - A[k])
                        if s <= 0:
                            t0, t1 = 1.0, 0.0
                        gap = min(gap, abs(s))
                    else:
                        a = (c[k] - A[k]) / d[k]
                        b = (c[k] + 1 - A[k]) / d[k]
                        if a > b:
                            a, b = b, a
                        t0, t1 = max(t0, a), min(t1, b)
                span = (t1 - t0) * float(np.linalg.norm(d))
                if span > margin and gap > 0:
                    res[(x, y, z)] = "in"
                elif span < -margin or gap <= 0 and span < margin:
                    res[(x, y, z)] = "out"
                else:
                    res[(x, y, z)] = "tie"
    return res


def test_traversal_matches_exact_geometry():
    """The FP32 traversal visits exactly the cells the segment passes through
    (brute force over every cell of a small grid), up to near ties."""
    rng = np.random.default_rng(7)
    ties = 0
    for _ in range(300):
        A = rng.uniform(-6, 6, size=3).astype(np.float32)
        B = (A + rng.uniform(-4, 4, size=3)).astype(np.float32)
        got = {tuple(v) for v in orc.traverse(A, B).tolist()}
        lo = np.floor(np.minimum(A, B)).astype(int) - 1
        hi = np.floor(np.maximum(A, B)).astype(int) + 2
        exact = _exact_cells(A, B, lo, hi, 1e-5)
        for cell, cls in exact.items():
            if cls == "in":
                assert cell in got, (A, B, cell)
            elif cls == "out":
                assert cell not in got, (A, B, cell)
            else:
                ties += 1
    assert ties < 50


def test_traversal_structure():
    """6-connected, monotone per axis, from floor(A) to floor(B), 1 + sum|di| voxels."""
    rng = np.random.default_rng(11)
    for _ in range(2000):
        A = rng.uniform(-1e3, 1e3, size=3).astype(np.float32)
        B = (A + rng.normal(0, 5, size=3)).astype(np.float32)
        v = orc.traverse(A, B)
        i0, i1 = np.floor(A).astype(int), np.floor(B).astype(int)
        assert (v[0] == i0).all() and (v[-1] == i1).all()
        assert len(v) == 1 + np.abs(i1 - i0).sum()
        steps = np.diff(v, axis=0)
        assert (np.abs(steps).sum(axis=1) == 1).all()
        for k in range(3):
            s = np.sign(i1[k] - i0[k])
            assert ((steps[:, k] * s) >= 0).all()


def test_axis_aligned_closed_form():
    """Along an axis the traversal is the integer range floor(A)..floor(B)."""
    for a, b in [(0.3, 7.9), (-3.5, 4.25), (10.75, -2.5), (-0.5, -0.25)]:
        v = orc.traverse([a, 2.5, -1.5], [b, 2.5, -1.5])
        ia, ib = math.floor(a), math.floor(b)
        step = 1 if ib >= ia else -1
        assert v[:, 0].tolist() == list(range(ia, ib + step, step))
        assert (v[:, 1] == 2).all() and (v[:, 2] == -2).all()


# ------------------------------------------------------------- distances
def test_axis_ray_hand_integration():
    g = _load("axis_ray_integration.json")
    vs, tr = g["voxel_size"], g["trunc"]
    T = np.array(g["T"], np.float32)

    def run(max_w, dropoff, frames):
        m = orc.OracleSubmap(vs, tr, max_w)
        for p in frames:
            m.integrate(np.array([p], np.float32), T, dropoff=dropoff, sensor=1)
        keys, D, W = m.extract()
        assert keys.tolist() == g["blocks"]
        out_d, out_w = [], []
        for x in g["voxels_x"]:
            b = [k for k, kk in enumerate(keys.tolist()) if kk == [x // 8, 0, 0]][0]
            out_d.append(D[b, x % 8])
            out_w.append(W[b, x % 8])
        return out_d, out_w

    cw = g["constant_weight"]
    d, w = run(1e4, 0, g["frames"][:1])
    assert d == cw["after_frame1"]["D"] and w == cw["after_frame1"]["W"]
    d, w = run(1e4, 0, g["frames"])
    assert d == cw["after_frame2"]["D"] and w == cw["after_frame2"]["W"]
    d, w = run(1.5, 0, g["frames"])
    assert d == cw["after_frame2_max_weight_1.5"]["D"] and w == cw["after_frame2_max_weight_1.5"]["W"]
    d, w = run(1e4, 1, g["frames"][:1])
    assert d == g["linear_dropoff_frame1"]["D"] and w == g["linear_dropoff_frame1"]["W"]


def test_distance_closed_form_oblique():
    """For a ray hitting a plane perpendicular to it, every band voxel's distance
    is the signed distance of its centre's projection on the ray to the plane:
    d = R - (c - o).u, which equals (p - c).u; checked via the plane equation."""
    rng = np.random.default_rng(3)
    vs, tr = 0.05, 0.15
    for _ in range(200):
        o = rng.uniform(-5, 5, size=3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        R = rng.uniform(0.5, 8)
        T = np.zeros(12, np.float32)
        T[[0, 5, 10]] = 1
        T[[3, 7, 11]] = o
        ps = (u * R).astype(np.float32)
        res = orc.point_obs(ps, T, vs, tr, sensor=1)
        vox, d, w, seg = res
        # the integrator transforms in FP32: with R = I, p = ps + t rounded once
        p = (ps + T[[3, 7, 11]]).astype(np.float64)
        o32 = T[[3, 7, 11]].astype(np.float64)
        uu = (p - o32) / np.linalg.norm(p - o32)
        c = (vox + 0.5) * np.float64(np.float32(vs))
        # plane through p with normal uu: signed distance of c's foot on the ray
        expect = np.clip(uu @ p - c @ uu, -np.float32(tr), np.float32(tr))
        assert np.allclose(d, expect, atol=1e-12)
        assert (np.abs(d) <= np.float32(tr)).all()
        assert (w == 1.0).all()


def test_quadratic_weight_closed_form():
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    for z in (0.5, 1.0, 2.0, 4.5):
        _, _, w, _ = orc.point_obs(np.array([0.1, -0.2, z], np.float32), T, 0.05, 0.15,
                                   weight_mode=1, sensor=0)
        assert np.allclose(w, 1.0 / np.float64(np.float32(z)) ** 2, rtol=1e-15)
        p = np.array([z, 0.3, -0.1], np.float32)
        _, _, w, _ = orc.point_obs(p, T, 0.05, 0.15, weight_mode=1, sensor=1)
        assert np.allclose(w, 1.0 / float(np.sum(p.astype(np.float64) ** 2)), rtol=1e-12)


def test_dropoff_closed_form():
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    vs, tr = 0.05, 0.15
    for mode in (1, 2):
        _, d, w, _ = orc.point_obs(np.array([0.0, 0.0, 2.0], np.float32), T, vs, tr, dropoff=mode)
        eps = np.float64(np.float32(vs))
        f = np.clip((np.float32(tr) + d) / (np.float32(tr) - eps), 0, None)
        f = np.where(d < -eps, f if mode == 1 else f * f, 1.0)
        assert np.allclose(w, f, rtol=1e-14)
        assert w.min() >= 0 and w.max() == 1.0


def test_invalid_points_and_key_range():
    m = orc.OracleSubmap(0.1, 0.3)
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    pts = np.array([[np.nan, 0, 1], [0, 0, 0.05], [0, 0, 100.0], [0, 0, 2.0]], np.float32)
    st = m.integrate(pts, T, max_range=50.0)
    assert st["valid"] == 1 and st["status"] == 0
    st = m.integrate(np.array([[0, 0, 2.0e6]], np.float32), T, max_range=1e9)
    assert st["status"] == -4 and st["key_range"] == 1


# ---------------------------------------------------- integration level
def _small_scan(seed=5, W=48, H=36, noise=0.01):
    scene = sg.room_scene(seed)
    cam = sg.Pinhole(W, H, 40.0, 40.0, (W - 1) / 2, (H - 1) / 2, 20.0, 1, noise)
    traj = sg.circle_trajectory(6)
    scans = [cam.render(scene, T, seed, k) for k, T in enumerate(traj)]
    poses = [np.ascontiguousarray(T.reshape(12), np.float32) for T in traj]
    return scene, scans, poses


def _integrate(scans, poses, vs=0.1, tr=0.3, max_w=1e4, **kw):
    m = orc.OracleSubmap(vs, tr, max_w, kw.pop("fp16", False))
    for s, T in zip(scans, poses):
        m.integrate(s, T, **kw)
    return m


def _brute_force_frame(points, T, vs, tr, vox_set):
    """Per voxel in vox_set x per point: does the band segment (FP64 geometry) pass
    through the voxel?  Returns sums and a mask of voxels with no near tie."""
    vs32, tr32 = np.float64(np.float32(vs)), np.float64(np.float32(tr))
    Tm = T.astype(np.float64).reshape(3, 4)
    swd = {v: 0.0 for v in vox_set}
    sw = {v: 0.0 for v in vox_set}
    tie = set()
    vox_arr = np.array(sorted(vox_set))
    for ps in points.astype(np.float32):
        if not np.isfinite(ps).all():
            continue
        # FP32 transform as the integrator performs it, then FP64 geometry
        p32 = np.zeros(3, np.float32)
        for k in range(3):
            a = np.float32(T[4 * k]) * ps[0]
            b = np.float32(T[4 * k + 1]) * ps[1]
            c = np.float32(T[4 * k + 2]) * ps[2]
            p32[k] = np.float32(np.float32(a + b) + c) + np.float32(T[4 * k + 3])
        p = p32.astype(np.float64)
        o = Tm[:, 3].astype(np.float32).astype(np.float64)
        r = p - o
        if not (0.1 <= np.linalg.norm(r) <= 1e9):
            continue
        u = r / np.linalg.norm(r)
        A, B = (p - tr32 * u) / vs32, (p + tr32 * u) / vs32
        lo = np.floor(np.minimum(A, B)).astype(int)
        hi = np.floor(np.maximum(A, B)).astype(int)
        sel = np.all((vox_arr >= lo) & (vox_arr <= hi), axis=1)
        for v in vox_arr[sel]:
            v = tuple(int(x) for x in v)
            cls = _exact_cells(A, B, v, (v[0] + 1, v[1] + 1, v[2] + 1), 1e-4)[v]
            if cls == "tie":
                tie.add(v)
            elif cls == "in":
                c = (np.array(v) + 0.5) * vs32
                d = float(np.clip((p - c) @ u, -tr32, tr32))
                swd[v] += d
                sw[v] += 1.0
    return swd, sw, tie


def test_brute_force_tiny_grid():
    """Two frames of a tiny scan: every voxel's D and W equal a brute-force
    enumeration of (voxel, point) pairs by exact geometry, then the merge."""
    scene, scans, poses = _small_scan(W=10, H=8)
    scans, poses = scans[:2], poses[:2]
    m = _integrate(scans, poses)
    keys, D, W = m.extract()
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    allv = {}
    for b, k in enumerate(keys):
        for l in range(512):
            lx, ly, lz = l % 8, (l // 8) % 8, l // 64
            allv[(k[0] * 8 + lx, k[1] * 8 + ly, k[2] * 8 + lz)] = (D[b, l], W[b, l])
    touched = {v for v, (dd, ww) in allv.items() if ww > 0}
    Dm = {v: 0.0 for v in touched}
    Wm = {v: 0.0 for v in touched}
    ties = set()
    for s, T in zip(scans, poses):
        swd, sw, tie = _brute_force_frame(s, T, 0.1, 0.3, touched)
        ties |= tie
        for v in touched:
            if sw[v] > 0:
                Dm[v] = (Dm[v] * Wm[v] + swd[v]) / (Wm[v] + sw[v])
                Wm[v] = Wm[v] + sw[v]
    checked = 0
    for v in touched - ties:
        assert abs(allv[v][1] - Wm[v]) < 1e-9, v
        assert abs(allv[v][0] - Dm[v]) < 1e-9, v
        checked += 1
    assert checked > 0.95 * len(touched) and checked > 200


def test_plane_head_on_matches_analytic_sdf():
    """Noise-free, narrow field of view, wall seen head on: D is the wall's
    signed distance within the small projective bias of the narrow cone."""
    scene = sg.Scene([(sg.SG_BOX, [4.0, -5.0, -5.0, 4.5, 5.0, 5.0])])
    cam = sg.Pinhole(64, 48, 600.0, 600.0, 31.5, 23.5, 20.0)
    T = sg.pose_from(sg.look_frame([1, 0, 0]), [0.0, 0.0, 0.0])
    pts = cam.render(scene, T, 1, 0)
    assert np.isfinite(pts).all()
    m = orc.OracleSubmap(0.05, 0.15)
    m.integrate(pts, np.float32(T.reshape(12)))
    keys, D, W = m.extract()
    b, l = np.nonzero(W > 0)
    v = keys[b] * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)
    c = (v + 0.5) * np.float64(np.float32(0.05))
    sdf = scene.sdf(c, 0.15)
    err = np.abs(D[b, l] - sdf)
    inside = np.abs(sdf) < 0.14
    assert err[inside].max() < 0.01
    assert (np.sign(D[b, l][np.abs(sdf) > 0.03]) == np.sign(sdf[np.abs(sdf) > 0.03])).all()


def test_repeat_frames_closed_form():
    """Noise-free static scan integrated k times with constant weight: D keeps
    the one-frame value; W = min(k m, max_weight) for m observations per frame."""
    scene, scans, poses = _small_scan(noise=0.0)
    s, T = scans[0], poses[0]
    m1 = _integrate([s], [T])
    k1, D1, W1 = m1.extract()
    for k, max_w in ((3, 1e4), (4, 5.0)):
        mk = _integrate([s] * k, [T] * k, max_w=max_w)
        kk, Dk, Wk = mk.extract()
        assert (kk == k1).all()
        assert np.allclose(Dk, D1, atol=1e-12)
        assert np.array_equal(Wk, np.minimum(k * W1, max_w))


def test_split_scan_equals_one_frame():
    """Weighted-mean associativity: a scan integrated as two half-scans (two
    frames) equals the one-frame result when the cap is not reached."""
    scene, scans, poses = _small_scan()
    s, T = scans[1], poses[1]
    one = _integrate([s], [T], weight_mode=1, sensor=0, dropoff=1)
    two = _integrate([s[::2], s[1::2]], [T, T], weight_mode=1, sensor=0, dropoff=1)
    k1, D1, W1 = one.extract()
    k2, D2, W2 = two.extract()
    assert (k1 == k2).all()
    assert np.allclose(W1, W2, rtol=1e-12, atol=0)
    assert np.allclose(D1, D2, atol=1e-12)


def test_point_order_invariance():
    scene, scans, poses = _small_scan()
    rng = np.random.default_rng(0)
    perm = [s[rng.permutation(len(s))] for s in scans]
    a = _integrate(scans, poses, weight_mode=1)
    b = _integrate(perm, poses, weight_mode=1)
    ka, Da, Wa = a.extract()
    kb, Db, Wb = b.extract()
    assert (ka == kb).all()
    assert np.allclose(Da, Db, atol=1e-12) and np.allclose(Wa, Wb, rtol=1e-12)


def test_invariants_over_frames():
    """|D| <= trunc, W never decreases, W <= max_weight."""
    scene, scans, poses = _small_scan()
    m = orc.OracleSubmap(0.1, 0.3, 7.0)
    prev = {}
    for s, T in zip(scans, poses):
        m.integrate(s, T)
        keys, D, W = m.extract()
        assert np.abs(D).max() <= np.float32(0.3)
        assert W.max() <= 7.0
        for b, k in enumerate(map(tuple, keys)):
            if k in prev:
                assert (W[b] >= prev[k]).all()
            prev[k] = W[b].copy()


def test_blocks_cover_all_band_voxels():
    """Every block holding a band voxel is allocated, even with zero weight."""
    scene, scans, poses = _small_scan()
    m = _integrate(scans[:1], poses[:1], dropoff=2)
    keys = {tuple(k) for k in m.extract()[0]}
    for ps in scans[0][::7]:
        r = orc.point_obs(ps, poses[0], 0.1, 0.3, dropoff=2)
        if r is None:
            continue
        for v in r[0]:
            assert tuple(int(x) // 8 for x in v) in keys


def test_block_set_and_sampled_agree_with_full():
    scene, scans, poses = _small_scan()
    m = _integrate(scans, poses, weight_mode=1, dropoff=1)
    keys, D, W = m.extract()
    bs = orc.block_set(scans, poses, 0.1, 0.3)
    assert (bs == keys).all()
    rng = np.random.default_rng(1)
    b = rng.integers(0, len(keys), 300)
    l = rng.integers(0, 512, 300)
    vox = keys[b] * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)
    Ds, Ws, _ = orc.sampled(scans, poses, vox, 0.1, 0.3, weight_mode=1, dropoff=1)
    assert np.array_equal(Ds, D[b, l]) and np.array_equal(Ws, W[b, l])


# ------------------------------------------------------------------ FP16
def test_round_half_matches_numpy():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0, 1, 10000), rng.uniform(-1, 1, 1000) * 1e-6,
                        rng.uniform(0, 1e4, 1000), [0.0, -0.0, 1.0, 65504.0, 2.0 ** -24]])
    assert np.array_equal(orc.round_half(x), x.astype(np.float16).astype(np.float64))


def test_fp16_mode_stores_half_values():
    scene, scans, poses = _small_scan()
    h = _integrate(scans, poses, fp16=True, weight_mode=1, sensor=0)
    f = _integrate(scans, poses, weight_mode=1, sensor=0)
    kh, Dh, Wh = h.extract()
    kf, Df, Wf = f.extract()
    assert (kh == kf).all()
    dn = Dh / np.float64(np.float32(0.3))
    assert np.array_equal(dn.astype(np.float16).astype(np.float64), dn)
    assert np.array_equal(Wh.astype(np.float16).astype(np.float64), Wh)
    # storage error vs the unrounded oracle stays within a few half ulps of trunc
    assert np.abs(Dh - Df).max() < 4 * 2.0 ** -11 * 0.3


# ------------------------------------------------------ free-space carving
def test_carving_axis_ray_closed_form():
    """A ray along +x from the sensor at x = 0.05 to a point at x = 1.05
    (vs 0.1, trunc 0.3): carving visits voxels 0..13 (floor((1.05 + 0.3) / 0.1)),
    the band only 7..13; in front of the band d = +trunc, inside it
    d = 1.05 - (i + 1/2) vs, clamped to +-trunc; weights 1."""
    vs, tr = 0.1, 0.3
    T = np.array([1, 0, 0, 0.05, 0, 1, 0, 0.05, 0, 0, 1, 0.05], np.float32)
    p = np.array([[1.0, 0.0, 0.0]], np.float32)            # submap x = 1.05
    out = {}
    for carve in (False, True):
        m = orc.OracleSubmap(vs, tr)
        st = m.integrate(p, T, sensor=1, carve=carve)
        keys, D, W = m.extract()
        xs = [int(k[0]) * 8 + l for k, b in zip(keys, range(len(keys))) for l in range(8) if W[b, l] > 0]
        out[carve] = (st, keys, D, W, sorted(xs))
    assert out[False][4] == list(range(7, 14)) and out[True][4] == list(range(0, 14))
    assert out[True][0]["obs"] == 14 and out[False][0]["obs"] == 7
    keys, D, W = out[True][1], out[True][2], out[True][3]
    for i in range(14):
        b = [j for j, k in enumerate(keys.tolist()) if k == [i // 8, 0, 0]][0]
        c = (np.float32(i) + 0.5) * np.float64(np.float32(vs))
        want = min(max(float(np.float32(1.05)) - c, -tr), tr)
        assert abs(D[b, i % 8] - want) < 1e-6 and W[b, i % 8] == 1.0


def test_carving_extends_the_band():
    """One ray: carving observes the band's voxels exactly as the band does and
    adds the voxels from the sensor to the band, all at d = +trunc."""
    rng = np.random.default_rng(7)
    T = np.array([1, 0, 0, 0.3, 0, 1, 0, -0.2, 0, 0, 1, 0.1], np.float32)
    for _ in range(5):
        p = np.array([rng.uniform(-1, 1, 2).tolist() + [rng.uniform(1.5, 3.0)]], np.float32)
        res = {}
        for carve in (False, True):
            m = orc.OracleSubmap(0.1, 0.3)
            m.integrate(p, T, carve=carve)
            keys, D, W = m.extract()
            res[carve] = {(tuple(k), l): (D[b, l], W[b, l]) for b, k in enumerate(keys.tolist())
                          for l in range(512) if W[b, l] > 0}
        band, carved = res[False], res[True]
        assert set(band) <= set(carved)
        assert all(carved[k] == band[k] for k in band)
        extra = [carved[k] for k in carved if k not in band]
        assert extra and all(abs(d - 0.3) < 1e-6 and w == 1.0 for d, w in extra)


def test_parallel_frame_sums_equal_sequential():
    """The OpenMP form of a frame (chunked per-thread sums added in chunk
    order) gives the sequential frame's blocks, counts and values up to FP64
    rounding of the sums' order (commutative sums, Sec. III-D)."""
    scene, scans, poses = _small_scan()
    a = orc.OracleSubmap(0.1, 0.3, 1e4)
    b = orc.OracleSubmap(0.1, 0.3, 1e4)
    for s, T in zip(scans, poses):
        sa = a.integrate(s, T, None, 1, 1)
        sb = b.integrate_parallel(s, T, 4, None, 1, 1)
        assert sa == sb
    ka, Da, Wa = a.extract()
    kb, Db, Wb = b.extract()
    assert np.array_equal(ka, kb)
    assert np.allclose(Da, Db, rtol=0, atol=1e-12) and np.allclose(Wa, Wb, rtol=1e-12, atol=0)
