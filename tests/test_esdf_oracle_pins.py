"""Pins of the ESDF oracle (CPU): the separable exact transform against brute
force, against a closed form (a plane of sites), against scipy's exact
Euclidean distance transform (an independent library routine), and the
field's invariants."""
import numpy as np
import pytest

from oracle import esdf as oe

VS = 0.1


def _random_submap(rng, nb=5, spread=2, p_site=0.02):
    keys = set()
    while len(keys) < nb:
        keys.add(tuple(rng.integers(-spread, spread + 1, 3)))
    keys = np.array(sorted(keys), np.int32)
    W = rng.uniform(0.5, 3.0, (nb, 512))
    W[rng.random((nb, 512)) < 0.3] = 0.0
    D = rng.uniform(0.5, 1.0, (nb, 512))
    s = rng.random((nb, 512)) < p_site
    D[s] = rng.uniform(-0.04, 0.04, s.sum())
    return keys, D, W


def test_edt1d_matches_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        f = np.where(rng.random(n) < 0.3, rng.integers(0, 500, n), oe.INF).astype(np.int64)
        got = oe.edt1d(f)
        q = np.arange(n)
        fin = f < oe.INF
        if not fin.any():
            assert (got == oe.INF).all()
            continue
        ref = ((q[:, None] - q[None, fin]) ** 2 + f[None, fin]).min(1)
        assert np.array_equal(got, ref)


def test_separable_matches_brute_force():
    rng = np.random.default_rng(1)
    for t in range(6):
        keys, D, W = _random_submap(rng, nb=int(rng.integers(1, 7)), p_site=[0.0, 0.002, 0.02, 0.2][t % 4])
        a = oe.esdf(keys, D, W, VS, 0.05, 0.0, 1.5)
        b = oe.esdf_bruteforce(keys, D, W, VS, 0.05, 0.0, 1.5)
        assert np.array_equal(a, b)


def test_plane_of_sites_closed_form():
    keys = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1]], np.int32)
    D = np.ones((5, 512))
    W = np.ones((5, 512))
    l = np.arange(512)
    vx = keys[:, 0:1] * 8 + (l % 8)[None, :]
    D[vx == 5] = 0.0                        # the plane x = 5 (voxel units)
    got = oe.esdf(keys, D, W, VS, 0.0, 0.0, 100.0)
    assert np.allclose(got, VS * np.abs(vx - 5), rtol=0, atol=1e-12)


def test_scipy_exact_edt_agrees():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    keys = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)], np.int32)
    D = np.ones((8, 512))
    W = np.ones((8, 512))
    site = rng.random((8, 512)) < 0.01
    D[site] = 0.0
    got = oe.esdf(keys, D, W, 1.0, 0.0, 0.0, 1e9)
    grid = np.ones((16, 16, 16), bool)   # True = not a site
    l = np.arange(512)
    for b, k in enumerate(keys):
        x, y, z = k[0] * 8 + l % 8, k[1] * 8 + (l // 8) % 8, k[2] * 8 + l // 64
        grid[x[site[b]], y[site[b]], z[site[b]]] = False
    ref = ndimage.distance_transform_edt(grid)
    for b, k in enumerate(keys):
        x, y, z = k[0] * 8 + l % 8, k[1] * 8 + (l // 8) % 8, k[2] * 8 + l // 64
        assert np.allclose(got[b], ref[x, y, z], rtol=1e-12, atol=1e-12)


def test_invariants_zero_at_sites_lipschitz_cap():
    rng = np.random.default_rng(3)
    keys, D, W = _random_submap(rng, nb=6, p_site=0.01)
    cap = 0.8
    e = oe.esdf(keys, D, W, VS, 0.05, 0.0, cap)
    s = oe.sites(D, W, 0.05, 0.0)
    assert (e[s] == 0).all() and (e[~s] > 0).all() and (e <= cap).all()
    # 1-Lipschitz between face neighbours inside a block (uncapped values)
    v = e.reshape(-1, 8, 8, 8)   # [b, z, y, x]
    for ax in (1, 2, 3):
        d = np.abs(np.diff(v, axis=ax))
        both = (np.delete(v, -1, axis=ax) < cap) & (np.delete(v, 0, axis=ax) < cap)
        assert (d[both] <= VS + 1e-12).all()


def test_no_sites_gives_cap():
    keys = np.array([[0, 0, 0], [3, -2, 1]], np.int32)
    D = np.ones((2, 512))
    W = np.ones((2, 512))
    assert (oe.esdf(keys, D, W, VS, 0.05, 0.0, 0.7) == 0.7).all()


def test_registration_points_and_bounds_by_hand():
    keys = np.array([[0, 0, 0], [-1, 2, 0]], np.int32)
    D = np.full((2, 512), 0.5)
    W = np.zeros((2, 512))
    D[0, 0], W[0, 0] = 0.01, 2.0          # voxel (0,0,0): taken
    D[0, 9], W[0, 9] = -0.02, 0.5         # voxel (1,1,0): W below w_min
    D[1, 64 + 7], W[1, 64 + 7] = 0.0, 1.0  # voxel (-8+7, 16, 1) = (-1, 16, 1): taken
    D[1, 3], W[1, 3] = 0.2, 5.0           # |D| above the band
    pts = oe.registration_points(keys, D, W, 0.1, 1.0, 0.05)
    want = np.array([[-0.05, 1.65, 0.15], [0.05, 0.05, 0.05]], np.float32)
    assert np.allclose(pts, want, rtol=0, atol=1e-7)
    assert np.allclose(oe.submap_bounds(keys, 0.1), [-0.8, 0.0, 0.0, 0.8, 2.4, 0.8], atol=1e-6)


# ------------------------------------------------------------- submap overlap
def _T(R=np.eye(3), t=(0, 0, 0)):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64)[:, None]], 1).reshape(12)


def test_overlap_identity_poses_closed_form():
    from oracle import esdf as oe
    a = [0, 0, 0, 2, 3, 4]
    b = [1, 1, 1, 5, 2, 2]
    v, box = oe.submap_overlap(a, _T(), b, _T())
    assert v == 1 * 1 * 1 and list(box) == [1, 1, 1, 2, 2, 2]
    v, _ = oe.submap_overlap(a, _T(), a, _T())
    assert v == 24.0                                     # a box with itself
    v, _ = oe.submap_overlap(a, _T(), b, _T(t=(10, 0, 0)))
    assert v == 0.0                                      # disjoint
    v, _ = oe.submap_overlap([0, 0, 0, 4, 4, 4], _T(), [1, 1, 1, 2, 2, 2], _T())
    assert v == 1.0                                      # containment: the smaller box
    v, _ = oe.submap_overlap([1, 1, 1, 0, 0, 0], _T(), a, _T())
    assert v == 0.0                                      # empty submap


def test_overlap_quarter_turn_and_translation():
    """A quarter turn about z maps the box x in [0,2], y in [0,1] to x in
    [-1,0], y in [0,2]; shifted by (+1, 0, 0) it overlaps [0,1]^2 x [0,1] in
    [0,1] x [0,1] x [0,1]."""
    from oracle import esdf as oe
    Rz = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    v, box = oe.submap_overlap([0, 0, 0, 2, 1, 1], _T(Rz, (1, 0, 0)), [0, 0, 0, 1, 1, 1], _T())
    assert abs(v - 1.0) < 1e-15 and np.allclose(box, [0, 0, 0, 1, 1, 1])
    # a 45 degree turn: the world box of the unit square spans sqrt(2)
    c = np.sqrt(0.5)
    v, box = oe.submap_overlap([0, 0, 0, 1, 1, 1], _T([[c, -c, 0], [c, c, 0], [0, 0, 1]]), [-5, -5, -5, 5, 5, 5],
                               _T())
    assert abs((box[3] - box[0]) - np.sqrt(2)) < 1e-12 and abs(v - 2.0) < 1e-12
