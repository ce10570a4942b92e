"""GPU parity of the submap ESDF against the oracle (exact squared distances
in voxel units, bit-exact; distances within FP32 rounding of the square
root), on fields the GPU integrator produced (so the ESDF kernels are tested
on their own: the oracle reads the same D and W)."""
import numpy as np
import pytest

import scenegen as sg
from _harness import int_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _integrate(wl, storage=0, pipelined=False, frames=None):
    import torch
    import paper_2410_21149_gb300 as cvx
    sm = wl.submaps[0]
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, storage, max_blocks=1 << 16, pipelined=pipelined)
    for sc in sm.scans[:frames]:
        sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, int_params(wl, sc))
    return sub


def _oracle_inputs(sub):
    """keys and the D, W the kernels see (float32, FP16 storage decoded the
    same way: half * trunc in float32)."""
    keys, D, W = (t.cpu().numpy() for t in sub.extract())
    if sub.storage == 1:
        D = D.astype(np.float32) * np.float32(sub.trunc)
        W = W.astype(np.float32)
    return keys, D.astype(np.float32), W.astype(np.float32)


def _sq_oracle(keys, D, W, band, w_min):
    """exact squared distances (voxel units) from the oracle's separable transform"""
    from oracle import esdf as oe
    e = oe.esdf(keys, D.astype(np.float64), W.astype(np.float64), 1.0, float(np.float32(band)), float(w_min), 1e12)
    return e


@pytest.mark.parametrize("storage,pipelined", [(0, False), (1, False), (0, True)])
def test_room_esdf_matches_oracle(storage, pipelined):
    wl = sg.make_c1(n_frames=4)
    sub = _integrate(wl, storage, pipelined)
    band, cap = sub.voxel_size, 1.5
    out, sq = sub.esdf(site_band=band, max_dist=cap, exact_sq=True)
    keys, D, W = _oracle_inputs(sub)
    ref = _sq_oracle(keys, D, W, band, 0.0)            # distances in voxel units, uncapped
    sq = sq.cpu().numpy().astype(np.float64)
    has = sq >= 0
    assert has.any() and (has == np.isfinite(ref) & (ref < 1e12)).all()
    assert np.array_equal(np.sqrt(sq[has]), ref[has])  # exact integers -> identical square roots
    o = out.cpu().numpy().astype(np.float64)
    expect = np.where(has, np.minimum(ref * np.float32(sub.voxel_size), cap), cap)
    assert np.abs(o - expect).max() <= 1e-6 * cap
    assert sub.status() == 0
    sub.close()


def test_multiroom_sampled_voxels_brute_force():
    """A larger field (multiroom frames): sampled voxels against brute force
    over every site."""
    wl = sg.make_c2(n_frames=6)
    sub = _integrate(wl)
    out, sq = sub.esdf(max_dist=3.0, exact_sq=True)
    keys, D, W = _oracle_inputs(sub)
    from oracle import esdf as oe
    site = oe.sites(D, W, np.float32(sub.voxel_size), 0.0)
    l = np.arange(512)
    idx = keys.astype(np.int64)[:, None, :] * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)[None]
    s = idx[site]
    rng = np.random.default_rng(0)
    pick = rng.choice(idx.shape[0] * 512, 400, replace=False)
    v = idx.reshape(-1, 3)[pick]
    d2 = ((v[:, None, :] - s[None, :, :]) ** 2).sum(-1).min(1)
    assert np.array_equal(sq.cpu().numpy().reshape(-1)[pick].astype(np.int64), d2)
    sub.close()


def test_no_sites_and_empty_submap():
    import torch
    import paper_2410_21149_gb300 as cvx
    sub = cvx.Submap(0.1, 0.3)
    assert sub.esdf().numel() == 0                     # no blocks: nothing to do
    pts = torch.tensor([[0.0, 0.0, 2.0]], device="cuda")
    sub.integrate(pts, np.eye(3, 4, dtype=np.float32), cvx.integrate_params())
    out, sq = sub.esdf(site_band=0.0, w_min=1e9, max_dist=0.9, exact_sq=True)   # no voxel qualifies
    assert (out == 0.9).all() and (sq == -1).all()
    with pytest.raises(cvx.CovoxError):
        sub.esdf(max_dist=0.0)
    sub.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_registration_points_and_bounds(storage):
    import torch
    from oracle import esdf as oe
    from paper_2410_21149_gb300 import _capi
    wl = sg.make_c1(n_frames=3)
    sub = _integrate(wl, storage)
    keys, D, W = _oracle_inputs(sub)
    w_min, band = 1.5, 0.05
    n = _capi.cvx_registration_points(sub.handle, w_min, band)          # count only
    xyz = torch.empty((n + 7, 3), dtype=torch.float32, device="cuda")
    assert _capi.cvx_registration_points(sub.handle, w_min, band, xyz) == n
    got = xyz[:n].cpu().numpy()
    got = got[np.lexsort((got[:, 2], got[:, 1], got[:, 0]))]
    want = oe.registration_points(keys, D, W, np.float32(sub.voxel_size), w_min, band)
    assert n > 100 and np.array_equal(got, want)
    small = torch.empty((10, 3), dtype=torch.float32, device="cuda")
    assert _capi.cvx_registration_points(sub.handle, w_min, band, small) == n   # count beyond capacity
    assert np.array_equal(_capi.cvx_submap_bounds(sub.handle), oe.submap_bounds(keys, np.float32(sub.voxel_size)))
    sub.close()


def test_submap_overlaps_match_oracle():
    """cvx_submap_overlaps on the bounds of real LiDAR submaps with their
    poses, plus rotated and empty ones, against the FP64 oracle (volumes
    within FP32 rounding of the transformed corners)."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from oracle import esdf as oe
    wl = sg.make_c3(n_scans=8, scans_per_submap=2, n_boxes=300)
    bounds, poses = [], []
    for sm in wl.submaps:
        sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, 0, max_blocks=1 << 14)
        for sc in sm.scans:
            sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor,
                          cvx.integrate_params(0, 0, wl.min_range, wl.max_range, 1, 64, 1024))
        bounds.append(cvx._capi.cvx_submap_bounds(sub.handle))
        poses.append(np.asarray(sm.T_world_sub, np.float32).reshape(12))
        sub.close()
    rng = np.random.default_rng(2)
    ang = rng.uniform(0, 2 * np.pi)
    R = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    bounds.append(bounds[0])
    poses.append(np.concatenate([R, np.asarray(poses[0]).reshape(3, 4)[:, 3:]], 1).reshape(12).astype(np.float32))
    bounds.append(np.array([1, 1, 1, 0, 0, 0], np.float32))          # empty submap
    poses.append(np.eye(3, 4, dtype=np.float32).reshape(12))
    B = torch.from_numpy(np.stack(bounds).astype(np.float32)).cuda()
    P = torch.from_numpy(np.stack(poses).astype(np.float32)).cuda()
    vol, boxes = cvx._capi.cvx_submap_overlaps(B, P, with_boxes=True)
    vol, boxes = vol.cpu().numpy(), boxes.cpu().numpy()
    n = len(bounds)
    nonzero = 0
    for i in range(n):
        for j in range(n):
            v, box = oe.submap_overlap(bounds[i], poses[i], bounds[j], poses[j])
            assert abs(vol[i, j] - v) <= 1e-5 * max(v, 1.0) + 1e-4, (i, j, vol[i, j], v)
            if v > 0:
                assert np.abs(boxes[i, j] - box).max() < 1e-4
                nonzero += 1
    assert nonzero >= n                        # at least every submap with itself
    assert vol[n - 1].max() == 0 and vol[:, n - 1].max() == 0
