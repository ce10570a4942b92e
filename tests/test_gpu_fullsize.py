"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on outputs the CPU oracle can compute at that size: the exact block set
of every checked submap, exact valid-point and observation counts, and D / W
of sampled voxels (the oracle restricted to the sample runs the same
definition over every point of every scan).

  - multiroom 640x480 x 200 frames, FP32, quadratic weight + linear drop-off,
    per-scan launches (the headline benchmark);
  - LiDAR 64x1024 x 2000 scans in 40 submaps through one batched persistent
    launch, checked on four of the submaps.
"""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from _harness import sort_blocks

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
W_REL, W_FLOOR = 1e-4, 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sample(keys, W, rng, n_pos=3000, n_zero=500):
    b, l = np.nonzero(W > 0)
    pick = rng.choice(len(b), min(n_pos, len(b)), replace=False)
    bz, lz = np.nonzero(W == 0)
    pz = rng.choice(len(bz), min(n_zero, len(bz)), replace=False) if len(bz) else np.zeros(0, int)
    bb = np.concatenate([b[pick], bz[pz]])
    ll = np.concatenate([l[pick], lz[pz]])
    vox = keys[bb].astype(np.int64) * 8 + np.stack([ll % 8, (ll // 8) % 8, ll // 64], 1)
    return bb, ll, vox.astype(np.int32)


def _check(keys, D, W, scans, poses, sensors, sm, wl, rng, weight_mode, dropoff):
    ko = orc.block_set(scans, poses, sm.voxel_size, sm.trunc, wl.min_range, wl.max_range, sensors)
    kg, Dg, Wg = sort_blocks(keys, D, W)
    assert np.array_equal(kg, ko), "block sets differ"
    bb, ll, vox = _sample(kg, Wg, rng)
    Do, Wo, _ = orc.sampled(scans, poses, vox, sm.voxel_size, sm.trunc, wl.max_weight, False, weight_mode,
                            dropoff, wl.min_range, wl.max_range, sensors)
    dg, wg = Dg[bb, ll], Wg[bb, ll]
    assert (np.abs(wg - Wo) <= W_REL * np.abs(Wo) + W_FLOOR).all()
    both = (Wo > W_FLOOR) & (wg > W_FLOOR)
    assert np.abs(dg - Do)[both].max() <= D_TOL
    return int(both.sum())


def test_multiroom_200_frames_full_size():
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c2()                       # 200 frames of 640x480
    sm = wl.submaps[0]
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, cvx.CVX_STORE_F32, max_blocks=1 << 18)
    prm = cvx.integrate_params(wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range, 0, 480, 640)
    for sc in sm.scans:
        sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, prm)
    keys, D, W = (t.cpu().numpy() for t in sub.extract())
    assert sub.status() == 0
    c = sub.counters()
    scans = [s.points for s in sm.scans]
    poses = [s.T_sub_sensor for s in sm.scans]
    n = _check(keys, D.astype(np.float64), W.astype(np.float64), scans, poses, None, sm, wl,
               np.random.default_rng(0), wl.weight_mode, wl.dropoff)
    assert n > 2500
    valid = sum(int((np.isfinite(s).all(1) & (s[:, 2] > 0)).sum()) for s in scans)   # range gate below
    assert c["frames"] == 200 and c["valid_points"] <= valid
    sub.close()


def test_lidar_2000_scans_batched_full_size():
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    wl = sg.make_c3()                       # 2000 scans, 40 submaps
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, cvx.CVX_STORE_F32, max_blocks=1 << 16)
            for sm in wl.submaps]
    keep, scans = [], []
    for m, sm in enumerate(wl.submaps):
        for sc in sm.scans:
            p = torch.from_numpy(sc.points).cuda()
            keep.append(p)
            scans.append((m, p, sc.T_sub_sensor, None,
                          cvx.integrate_params(0, 0, wl.min_range, wl.max_range, 1, 64, 1024, 256, -1)))
    b = _capi.cvx_batch_create(len(subs), len(scans))
    _capi.cvx_integrate_batch(b, [s.handle for s in subs], scans)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(b) == 0
    rng = np.random.default_rng(1)
    checked = 0
    for m in (0, 13, 26, 39):
        sm, sub = wl.submaps[m], subs[m]
        assert sub.status() == 0
        keys, D, W = (t.cpu().numpy() for t in sub.extract())
        pts = [s.points for s in sm.scans]
        poses = [s.T_sub_sensor for s in sm.scans]
        checked += _check(keys, D.astype(np.float64), W.astype(np.float64), pts, poses, [1] * len(pts), sm, wl,
                          rng, 0, 0)
        c = sub.counters()
        assert c["frames"] == len(sm.scans)
    assert checked > 8000
    _capi.cvx_batch_destroy(b)
    for s in subs:
        s.close()


def test_batched_32_submaps_fp16_full_size():
    """The batched workload at full size, as bench.py times it: 32 submaps of
    1-16 scans mixing 640x480 pinhole frames and 64x1024 LiDAR scans, voxel
    sizes 0.05 / 0.10 / 0.20 m, FP16 storage, pipelined submaps, one batched
    persistent launch (256-point tiles, two shared block slots).  Every
    submap's block set bit-exact; 3,000 sampled voxels per submap against the
    oracle's FP16 storage mode (D within 1e-3 trunc, W within one half ulp)."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    wl = sg.make_c4()
    assert len(wl.submaps) == 32
    assert {s.width for sm in wl.submaps for s in sm.scans} == {640, 1024}
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, cvx.CVX_STORE_F16, max_blocks=1 << 16,
                       pipelined=True) for sm in wl.submaps]
    keep, scans = [], []
    k = 0
    while any(k < len(sm.scans) for sm in wl.submaps):
        for m, sm in enumerate(wl.submaps):
            if k < len(sm.scans):
                sc = sm.scans[k]
                p = torch.from_numpy(sc.points).cuda()
                keep.append(p)
                scans.append((m, p, sc.T_sub_sensor, None,
                              cvx.integrate_params(0, 0, wl.min_range, wl.max_range, sc.sensor, sc.height,
                                                   sc.width, 256, 2)))
        k += 1
    b = _capi.cvx_batch_create(len(subs), len(scans))
    _capi.cvx_integrate_batch(b, [s.handle for s in subs], scans)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(b) == 0
    rng = np.random.default_rng(4)
    checked = 0
    for m, (sm, sub) in enumerate(zip(wl.submaps, subs)):
        assert sub.status() == 0
        keys, D, W = (t.cpu().numpy() for t in sub.extract())
        D = D.astype(np.float64) * np.float64(np.float32(sm.trunc))
        W = W.astype(np.float64)
        pts = [s.points for s in sm.scans]
        poses = [s.T_sub_sensor for s in sm.scans]
        sensors = [s.sensor for s in sm.scans]
        ko = orc.block_set(pts, poses, sm.voxel_size, sm.trunc, wl.min_range, wl.max_range, sensors)
        kg, Dg, Wg = sort_blocks(keys, D, W)
        assert np.array_equal(kg, ko), f"block sets differ (submap {m})"
        bb, ll, vox = _sample(kg, Wg, rng)
        Do, Wo, _ = orc.sampled(pts, poses, vox, sm.voxel_size, sm.trunc, wl.max_weight, True, 0, 0,
                                wl.min_range, wl.max_range, sensors)
        dg, wg = Dg[bb, ll], Wg[bb, ll]
        ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(Wo), 2.0 ** -14))) - 10)
        assert (np.abs(wg - Wo) <= ulp + W_FLOOR).all(), f"W (submap {m})"
        both = (Wo > W_FLOOR) & (wg > W_FLOOR)
        assert np.abs(dg - Do)[both].max() <= 1e-3 * sm.trunc, f"D (submap {m})"
        assert both.sum() >= min(3000, int((Wg > 0).sum()))
        checked += int(both.sum())
        assert sub.counters()["frames"] == len(sm.scans)
    assert checked > 32 * 2500
    _capi.cvx_batch_destroy(b)
    for s in subs:
        s.close()
