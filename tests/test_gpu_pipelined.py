"""The pipelined per-scan path (submaps created with CVX_SUBMAP_PIPELINED):
each integrate call accumulates its scan and merges the previous call's scan
in one launch.  Results must equal the oracle's frame-by-frame
aggregate-then-merge (Sec. III-D) whatever the scheduling: pending scans
merged by flush, extract, counters or a batched launch, dropped by reset,
and recorded CUDA graphs replayed.  Same tolerances as the plain path."""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, int_params, run_gpu, run_oracle, sort_blocks

pytestmark = pytest.mark.gpu

D_TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _host(sub, storage, trunc):
    keys, D, W = (t.cpu().numpy() for t in sub.extract())
    D = D.astype(np.float64)
    if storage == 1:
        D = D * np.float64(np.float32(trunc))
    return keys, D, W.astype(np.float64)


def test_room_10_frames_fp32():
    wl = sg.make_c1()
    g, o = run_gpu(wl, pipelined=True)[0], run_oracle(wl)[0]
    r = compare(g, o, D_TOL_F32)
    cnt, tot = g[3], o[3]
    assert cnt["frames"] == 10
    assert cnt["valid_points"] == tot["valid"] and cnt["observations"] == tot["obs"]
    assert cnt["blocks_touched"] == tot["blocks"]
    assert r["voxels"] > 30000


@pytest.mark.parametrize("dropoff,lb", [(1, 0), (2, 4), (0, -1)])
def test_multiroom_fp32(dropoff, lb):
    wl = sg.make_c2(n_frames=3, dropoff=dropoff)
    compare(run_gpu(wl, pipelined=True, local_blocks=lb)[0], run_oracle(wl)[0], D_TOL_F32)


def test_multiroom_fp16_storage():
    wl = sg.make_c2(n_frames=4, storage=1)
    tr = wl.submaps[0].trunc
    compare(run_gpu(wl, pipelined=True)[0], run_oracle(wl, fp16=True)[0], 1e-3 * tr, fp16_trunc=tr)


def test_lidar_submaps_fp32():
    wl = sg.make_c3(n_scans=6, scans_per_submap=3, n_boxes=400)
    for a, b in zip(run_gpu(wl, pipelined=True, local_blocks=-1), run_oracle(wl)):
        compare(a, b, D_TOL_F32)


def test_pending_scan_flush_extract_and_continue():
    """Counters after every call; extract in the middle (merges the pending
    scan early) and continue; flush twice is a no-op."""
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c1(n_frames=6)
    sm = wl.submaps[0]
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, pipelined=True)
    for k, sc in enumerate(sm.scans):
        sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, int_params(wl, sc))
        if k == 2:
            sub.extract()
        assert sub.counters()["frames"] == k + 1
    sub.flush()
    sub.flush()
    keys, D, W = _host(sub, 0, sm.trunc)
    c = sub.counters()
    o = run_oracle(wl)[0]
    compare((keys, D, W, c, sub.status()), o, D_TOL_F32)
    assert c["frames"] == 6 and c["observations"] == o[3]["obs"] and c["blocks_touched"] == o[3]["blocks"]
    sub.close()


def test_reset_drops_pending_scan():
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c1(n_frames=4)
    sm = wl.submaps[0]
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, pipelined=True)
    pts = [torch.from_numpy(s.points).cuda() for s in sm.scans]
    for p, sc in zip(pts[:3], sm.scans[:3]):      # three scans, the last left pending
        sub.integrate(p, sc.T_sub_sensor, int_params(wl, sc))
    sub.reset()
    for p, sc in zip(pts, sm.scans):
        sub.integrate(p, sc.T_sub_sensor, int_params(wl, sc))
    keys, D, W = _host(sub, 0, sm.trunc)
    c = sub.counters()
    assert c["frames"] == 4
    compare((keys, D, W, c, sub.status()), run_oracle(wl)[0], D_TOL_F32)
    sub.close()


def test_graph_capture_replay():
    """reset + every scan + flush recorded once, replayed twice: the set
    parity lives on the device, so each replay equals one eager pass."""
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c2(n_frames=3, width=320, height=240)
    sm = wl.submaps[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, pipelined=True, stream=stream)
        pts = [torch.from_numpy(s.points).cuda() for s in sm.scans]
        prm = [int_params(wl, s) for s in sm.scans]
        sub.integrate(pts[0], sm.scans[0].T_sub_sensor, prm[0], stream=stream)   # warm-up, left pending
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sub.reset(stream=stream)
        for p, sc, q in zip(pts, sm.scans, prm):
            sub.integrate(p, sc.T_sub_sensor, q, stream=stream)
        sub.flush(stream=stream)
    o = run_oracle(wl)[0]
    for _ in range(2):
        with torch.cuda.stream(stream):
            g.replay()
        stream.synchronize()
        keys, D, W = _host(sub, 0, sm.trunc)
        c = sub.counters()
        assert c["frames"] == 3
        compare((keys, D, W, c, sub.status()), o, D_TOL_F32)
    sub.close()


def test_per_scan_then_batched():
    """The first scans per scan (the last one left pending), the rest in one
    batched launch over the same pipelined submaps."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    wl = sg.make_c3(n_scans=6, scans_per_submap=3, n_boxes=300)
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, pipelined=True) for sm in wl.submaps]
    keep, rest = [], []
    for m, (sm, sub) in enumerate(zip(wl.submaps, subs)):
        for k, sc in enumerate(sm.scans):
            p = torch.from_numpy(sc.points).cuda()
            keep.append(p)
            prm = int_params(wl, sc)
            if k < 2:
                sub.integrate(p, sc.T_sub_sensor, prm)
            else:
                rest.append((m, p, sc.T_sub_sensor, None, prm))
    b = _capi.cvx_batch_create(len(subs), len(rest))
    _capi.cvx_integrate_batch(b, [s.handle for s in subs], rest)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(b) == 0
    for sm, sub, o in zip(wl.submaps, subs, run_oracle(wl)):
        keys, D, W = _host(sub, 0, sm.trunc)
        c = sub.counters()
        assert c["frames"] == len(sm.scans)
        compare((keys, D, W, c, sub.status()), o, D_TOL_F32)
    _capi.cvx_batch_destroy(b)
    for s in subs:
        s.close()


def test_pipelined_equals_plain_submap():
    """The same scans through a plain and a pipelined submap: identical block
    sets, D and W within the parity tolerances of each other."""
    wl = sg.make_c2(n_frames=4, width=320, height=240)
    a = run_gpu(wl)[0]
    b = run_gpu(wl, pipelined=True)[0]
    ka, Da, Wa = sort_blocks(a[0], a[1], a[2])
    kb, Db, Wb = sort_blocks(b[0], b[1], b[2])
    assert np.array_equal(ka, kb)
    assert (np.abs(Wa - Wb) <= 1e-4 * np.abs(Wa) + 1e-6).all()
    m = (Wa > 1e-6) & (Wb > 1e-6)
    assert np.abs(Da - Db)[m].max() <= D_TOL_F32
    assert a[3] == b[3]


def test_capacity_error_skips_only_that_scan():
    """A scan that overflows the pool is not merged (voxels unchanged) but the
    error is sticky; in the pipelined path the skip happens one launch later."""
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c1(n_frames=2)
    sub = cvx.Submap(0.1, 0.3, max_blocks=8, hash_slots=16, pipelined=True)
    s = wl.submaps[0].scans[0]
    sub.integrate(torch.from_numpy(s.points).cuda(), s.T_sub_sensor, cvx.integrate_params())
    assert sub.status() == cvx._capi.CVX_ERR_CAPACITY      # seen while the scan is pending
    keys, D, W = sub.extract()
    assert len(keys) == 8 and float(W.abs().max()) == 0.0 and float(D.abs().max()) == 0.0
    assert sub.status() == cvx._capi.CVX_ERR_CAPACITY      # sticky after the merge pass
    assert sub.counters()["frames"] == 1


def test_key_range_error():
    import torch
    import paper_2410_21149_gb300 as cvx
    sub = cvx.Submap(0.1, 0.3, pipelined=True)
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    bad = torch.tensor([[0.0, 0.0, 2.0], [0.0, 0.0, 2.0e6]], device="cuda")
    good = torch.tensor([[0.0, 0.0, 2.0]], device="cuda")
    sub.integrate(bad, T, cvx.integrate_params(max_range=1e9))
    sub.integrate(good, T, cvx.integrate_params(max_range=1e9))   # merges the bad scan (skipped)
    sub.flush()
    assert sub.status() == cvx._capi.CVX_ERR_KEY_RANGE
    keys, D, W = sub.extract()
    import oracle as orc
    om = orc.OracleSubmap(0.1, 0.3)
    om.integrate(np.array([[0.0, 0.0, 2.0]], np.float32), T)
    ko, Do, Wo = om.extract()
    kg, Dg, Wg = sort_blocks(keys.cpu().numpy(), D.cpu().double().numpy(), W.cpu().double().numpy())
    assert np.array_equal(kg, ko)       # only the good scan's voxels carry weight
    assert np.array_equal(Wg, Wo) and np.abs(Dg - Do).max() < D_TOL_F32
    assert sub.counters()["frames"] == 2
