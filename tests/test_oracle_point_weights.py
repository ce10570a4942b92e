"""Pins of the oracle's per-point weights (CPU only).

The weighting paragraph of coVoxSLAM Sec. III-C lets every ray carry its own
weight (the learned weight of this library is one).  What pins the oracle's
per-point mode: it reduces to the constant mode for unit weights, uniform
power-of-two weights scale W exactly and leave D unchanged (the weighted mean
is scale invariant), weights of 1/z^2 reproduce the quadratic mode, two rays
meeting in a voxel give the closed-form weighted mean of their distances, and
an invalid weight (NaN, infinite or negative) drops its point entirely.
"""
import numpy as np

import oracle as orc
import scenegen as sg


def _scans(seed=7, W=48, H=36, n=3):
    scene = sg.room_scene(seed)
    cam = sg.Pinhole(W, H, 40.0, 40.0, (W - 1) / 2, (H - 1) / 2, 20.0, 1, 0.01)
    traj = sg.circle_trajectory(n)
    scans = [cam.render(scene, T, seed, k) for k, T in enumerate(traj)]
    poses = [np.ascontiguousarray(T.reshape(12), np.float32) for T in traj]
    return scans, poses


def _run(scans, poses, pws=None, weight_mode=2, dropoff=0, vs=0.1, tr=0.3, max_w=1e6):
    m = orc.OracleSubmap(vs, tr, max_w)
    stats = []
    for k, (s, T) in enumerate(zip(scans, poses)):
        stats.append(m.integrate(s, T, None if pws is None else pws[k], weight_mode, dropoff, 0.1, 20.0, 0))
    return m.extract(), stats


def test_unit_weights_equal_constant_mode():
    scans, poses = _scans()
    (k1, D1, W1), _ = _run(scans, poses, None, weight_mode=0)
    (k2, D2, W2), _ = _run(scans, poses, [np.ones(len(s), np.float32) for s in scans])
    assert np.array_equal(k1, k2) and np.array_equal(D1, D2) and np.array_equal(W1, W2)


def test_power_of_two_weights_scale_w_exactly():
    scans, poses = _scans()
    (k1, D1, W1), _ = _run(scans, poses, None, weight_mode=0, dropoff=1)
    for e in (-7, 5):
        c = np.float32(2.0 ** e)
        (k2, D2, W2), _ = _run(scans, poses, [np.full(len(s), c, np.float32) for s in scans], dropoff=1)
        assert np.array_equal(k1, k2)
        assert np.array_equal(D1, D2)          # the weighted mean does not see a common scale
        assert np.array_equal(W2, W1 * float(c))


def test_inverse_square_depth_weights_match_quadratic_mode():
    scans, poses = _scans()
    pws = []
    for s in scans:
        z = s[:, 2].astype(np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            pws.append(np.where(np.isfinite(z) & (z > 0), 1.0 / (z * z), 1.0).astype(np.float32))
    (k1, D1, W1), _ = _run(scans, poses, None, weight_mode=1, dropoff=1)
    (k2, D2, W2), _ = _run(scans, poses, pws, dropoff=1)
    assert np.array_equal(k1, k2)
    assert np.allclose(W2, W1, rtol=2e-7, atol=0)   # float32 rounding of each 1/z^2
    # each weight moves by at most 2^-24 relative, so each weighted mean of
    # distances in [-trunc, trunc] moves by at most 2 * 2^-24 * 2 trunc
    assert np.abs(D2 - D1).max() < 2 * 2.0 ** -24 * 2 * 0.3


def test_two_rays_weighted_mean_closed_form():
    """Two points on one ray, 6 cm apart, whose bands share voxels: a shared
    voxel holds (a d1 + b d2) / (a + b) with weight a + b; a voxel of one band
    only holds that point's distance and weight."""
    T = np.array([1, 0, 0, 0.013, 0, 1, 0, 0.021, 0, 0, 1, 0.007], np.float32)
    p1 = np.array([0.031, 0.017, 2.0], np.float32)
    p2 = (p1 * np.float32(1.03)).astype(np.float32)
    a, b = np.float32(0.75), np.float32(3.5)
    vs, tr = 0.05, 0.15
    o1 = orc.point_obs(p1, T, vs, tr)
    o2 = orc.point_obs(p2, T, vs, tr)
    m = orc.OracleSubmap(vs, tr, 1e6)
    m.integrate(np.stack([p1, p2]), T, np.array([a, b], np.float32), 2, 0, 0.1, 20.0, 0)
    keys, D, W = m.extract()
    where = {tuple(k): q for q, k in enumerate(keys)}

    def at(v):
        blk = tuple(int(x) for x in np.floor_divide(v, 8))
        loc = v - 8 * np.floor_divide(v, 8)
        q = where[blk]
        li = int(loc[0] + 8 * loc[1] + 64 * loc[2])
        return D[q, li], W[q, li]

    d1 = {tuple(v): d for v, d in zip(o1[0], o1[1])}
    d2 = {tuple(v): d for v, d in zip(o2[0], o2[1])}
    shared = set(d1) & set(d2)
    assert len(shared) >= 2 and len(set(d1) ^ set(d2)) >= 1
    for v in set(d1) | set(d2):
        Dv, Wv = at(np.array(v))
        if v in shared:
            expect = (float(a) * d1[v] + float(b) * d2[v]) / (float(a) + float(b))
            assert abs(Dv - expect) < 1e-15 and Wv == float(a) + float(b)
        elif v in d1:
            assert abs(Dv - d1[v]) < 1e-15 and Wv == float(a)
        else:
            assert abs(Dv - d2[v]) < 1e-15 and Wv == float(b)


def test_invalid_weights_drop_their_points():
    scans, poses = _scans()
    rng = np.random.default_rng(3)
    pws, kept = [], []
    for s in scans:
        w = rng.uniform(0.1, 4.0, len(s)).astype(np.float32)
        bad = rng.choice(len(s), len(s) // 10, replace=False)
        w[bad[0::3]] = np.nan
        w[bad[1::3]] = np.inf
        w[bad[2::3]] = -1.5
        keep = np.ones(len(s), bool)
        keep[bad] = False
        pws.append(w)
        kept.append(keep)
    (k1, D1, W1), st1 = _run(scans, poses, pws)
    (k2, D2, W2), st2 = _run([s[m] for s, m in zip(scans, kept)], poses, [w[m] for w, m in zip(pws, kept)])
    assert np.array_equal(k1, k2) and np.array_equal(D1, D2) and np.array_equal(W1, W2)
    assert [a["valid"] for a in st1] == [b["valid"] for b in st2]
    # the block set and the sampled voxels see the same rule
    bs = orc.block_set(scans, poses, 0.1, 0.3, 0.1, 20.0, point_weights=pws)
    assert np.array_equal(bs, k1)
    b, l = np.nonzero(W1 > 0)
    pick = rng.choice(len(b), 200, replace=False)
    vox = k1[b[pick]].astype(np.int64) * 8 + np.stack([l[pick] % 8, (l[pick] // 8) % 8, l[pick] // 64], 1)
    Ds, Ws, _ = orc.sampled(scans, poses, vox.astype(np.int32), 0.1, 0.3, 1e6, False, 2, 0, 0.1, 20.0,
                            point_weights=pws)
    assert np.allclose(Ds, D1[b[pick], l[pick]], atol=1e-12) and np.allclose(Ws, W1[b[pick], l[pick]], rtol=1e-12)


def test_zero_weight_point_still_allocates():
    """A zero weight is valid: its band's blocks are allocated, nothing is merged."""
    T = np.array([1, 0, 0, 0.0, 0, 1, 0, 0.0, 0, 0, 1, 0.0], np.float32)
    p = np.array([[0.2, 0.1, 3.0]], np.float32)
    m = orc.OracleSubmap(0.1, 0.3, 1e4)
    st = m.integrate(p, T, np.zeros(1, np.float32), 2, 0, 0.1, 20.0, 0)
    keys, D, W = m.extract()
    assert st["valid"] == 1 and len(keys) >= 1 and (W == 0).all() and (D == 0).all()
