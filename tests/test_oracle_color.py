"""Pins of the oracle's colour integration (CPU only).

The paper times "TSDF + Color" integration (Sec. IV, TSDF results): every
voxel also fuses the points' colours.  Reading: each observation carries its
point's colour with the observation's weight, and the colour follows the
same weighted running mean as the distance, C <- (C W + S_wc) / (W + S_w)
(uncapped denominator, like D).  Pins: a wall of one colour reproduces that
colour in every observed voxel; two points of different colours meeting in a
voxel give the closed-form weighted mean; colours change neither D nor W;
per-channel linearity.
"""
import numpy as np

import oracle as orc
import scenegen as sg


def _scans(seed=9, W=40, H=30, n=3):
    scene = sg.room_scene(seed)
    cam = sg.Pinhole(W, H, 35.0, 35.0, (W - 1) / 2, (H - 1) / 2, 20.0, 1, 0.01)
    traj = sg.circle_trajectory(n)
    scans = [cam.render(scene, T, seed, k) for k, T in enumerate(traj)]
    poses = [np.ascontiguousarray(T.reshape(12), np.float32) for T in traj]
    return scans, poses


def _run(scans, poses, cols, weight_mode=1, dropoff=1, max_w=1e4):
    m = orc.OracleSubmap(0.1, 0.3, max_w)
    for s, T, c in zip(scans, poses, cols):
        m.integrate(s, T, None, weight_mode, dropoff, 0.1, 20.0, 0, colors=c)
    k, D, W = m.extract()
    return k, D, W, m.extract_colors()


def test_single_colour_reproduced_exactly():
    scans, poses = _scans()
    c = np.array([0.25, 0.5, 0.875], np.float32)
    k, D, W, C = _run(scans, poses, [np.tile(c, (len(s), 1)) for s in scans], max_w=3.0)   # the cap is met
    m = W > 0
    for ch in range(3):
        assert np.abs(C[:, ch, :][m] - float(c[ch])).max() < 1e-14
        assert (C[:, ch, :][~m] == 0).all()


def test_colour_leaves_distance_and_weight_unchanged():
    scans, poses = _scans()
    rng = np.random.default_rng(1)
    k0, D0, W0 = _run(scans, poses, [None] * len(scans))[:3]
    k1, D1, W1, _ = _run(scans, poses, [rng.uniform(0, 1, (len(s), 3)).astype(np.float32) for s in scans])
    assert np.array_equal(k0, k1) and np.array_equal(D0, D1) and np.array_equal(W0, W1)


def test_two_points_weighted_mean_of_colours():
    T = np.array([1, 0, 0, 0.013, 0, 1, 0, 0.021, 0, 0, 1, 0.007], np.float32)
    p1 = np.array([0.031, 0.017, 2.0], np.float32)
    p2 = (p1 * np.float32(1.03)).astype(np.float32)   # same ray, bands overlap
    c1 = np.array([1.0, 0.0, 0.5], np.float32)
    c2 = np.array([0.0, 1.0, 0.25], np.float32)
    w = np.array([0.75, 3.5], np.float32)
    m = orc.OracleSubmap(0.05, 0.15, 1e6)
    m.integrate(np.stack([p1, p2]), T, w, 2, 0, 0.1, 20.0, 0, colors=np.stack([c1, c2]))
    keys, D, W = m.extract()
    C = m.extract_colors()
    o1 = {tuple(v) for v in orc.point_obs(p1, T, 0.05, 0.15)[0]}
    o2 = {tuple(v) for v in orc.point_obs(p2, T, 0.05, 0.15)[0]}
    where = {tuple(k): q for q, k in enumerate(keys)}
    shared = o1 & o2
    assert len(shared) >= 2
    for v in o1 | o2:
        v = np.array(v)
        q = where[tuple(int(x) for x in np.floor_divide(v, 8))]
        loc = v - 8 * np.floor_divide(v, 8)
        li = int(loc[0] + 8 * loc[1] + 64 * loc[2])
        if tuple(v) in shared:
            expect = (0.75 * c1.astype(np.float64) + 3.5 * c2.astype(np.float64)) / 4.25
        elif tuple(v) in o1:
            expect = c1.astype(np.float64)
        else:
            expect = c2.astype(np.float64)
        assert np.abs(C[q, :, li] - expect).max() < 1e-14


def test_colour_is_linear_per_channel():
    """Fused colour of a*c + b is a*C + b (the weighted mean is affine);
    colours on a 2^-10 grid, so a*c + b is exact in float32 too."""
    scans, poses = _scans()
    rng = np.random.default_rng(4)
    cols = [(rng.integers(0, 1024, (len(s), 3)) / 1024.0).astype(np.float32) for s in scans]
    _, _, W, C = _run(scans, poses, cols)
    _, _, _, C2 = _run(scans, poses, [(0.5 * c + 0.25).astype(np.float32) for c in cols])
    m = np.broadcast_to((W > 0)[:, None, :], C.shape)
    assert np.abs(C2[m] - (0.5 * C[m] + 0.25)).max() < 1e-12


def test_non_finite_colour_drops_its_point():
    """A point with a NaN or infinite colour channel is skipped: the run equals
    the run without those points, in D, W, C and the valid-point count."""
    scans, poses = _scans()
    rng = np.random.default_rng(5)
    cols = [rng.uniform(0, 1, (len(s), 3)).astype(np.float32) for s in scans]
    bad = []
    for c in cols:
        b = rng.choice(len(c), len(c) // 10, replace=False)
        c[b[0::3], 0] = np.nan
        c[b[1::3], 1] = np.inf
        c[b[2::3], 2] = -np.inf
        bad.append(b)
    m1 = orc.OracleSubmap(0.1, 0.3, 1e4)
    m2 = orc.OracleSubmap(0.1, 0.3, 1e4)
    v1 = v2 = 0
    for s, T, c, b in zip(scans, poses, cols, bad):
        v1 += m1.integrate(s, T, None, 1, 1, 0.1, 20.0, 0, colors=c)["valid"]
        keep = np.setdiff1d(np.arange(len(s)), b)
        v2 += m2.integrate(s[keep], T, None, 1, 1, 0.1, 20.0, 0, colors=c[keep])["valid"]
    assert v1 == v2 and v1 > 0
    for a, b in zip(m1.extract() + (m1.extract_colors(),), m2.extract() + (m2.extract_colors(),)):
        assert np.array_equal(a, b)
