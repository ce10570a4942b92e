"""Batched persistent integration (many submaps, uneven mixed scans, one
persistent launch working through a queue of tile and merge items) against
the CPU oracle and the per-scan path."""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, run_gpu, run_gpu_batched, run_oracle, sort_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def mixed():
    return sg.make_c4(n_submaps=6, max_scans=4, depth_wh=(160, 120), lidar_rc=(16, 256))


@pytest.mark.parametrize("pipelined,wave_limit,sets", [(False, 0, 0), (True, 0, 0), (True, 2, 0), (True, 0, 4),
                                                        (True, 3, 4)])
def test_batched_mixed_fp32_fp16_vs_oracle(mixed, pipelined, wave_limit, sets):
    """Mixed storage; one, two and four per-scan sets (a scan's tiles overlap
    the merges of the previous one or three scans of its submap), and rounds
    cut into chunks of two or three scans."""
    storages = [m % 2 for m in range(len(mixed.submaps))]
    g = run_gpu_batched(mixed, storages, pipelined=pipelined, wave_limit=wave_limit, sets=sets)
    for m, (a, st) in enumerate(zip(g, storages)):
        sm = mixed.submaps[m]
        sub = sg.Workload(mixed.name, [sm], mixed.max_weight, mixed.weight_mode, mixed.dropoff,
                          mixed.min_range, mixed.max_range, mixed.scene, st)
        o = run_oracle(sub, fp16=bool(st))[0]
        if st:
            compare(a, o, 1e-3 * sm.trunc, fp16_trunc=sm.trunc)
        else:
            compare(a, o, 1e-5)
        assert a[3]["frames"] == len(sm.scans)
        assert a[3]["observations"] == o[3]["obs"]


@pytest.mark.parametrize("parts", [1, 7, 256])
def test_merge_parts_do_not_change_results(mixed, parts):
    """Each scan's merge cut into 1, 7 or 256 work items (the most the
    launch allows): the same submaps as the oracle's."""
    storages = [m % 2 for m in range(len(mixed.submaps))]
    g = run_gpu_batched(mixed, storages, sets=4, merge_parts=parts)
    for m, (a, st) in enumerate(zip(g, storages)):
        sm = mixed.submaps[m]
        sub = sg.Workload(mixed.name, [sm], mixed.max_weight, mixed.weight_mode, mixed.dropoff,
                          mixed.min_range, mixed.max_range, mixed.scene, st)
        o = run_oracle(sub, fp16=bool(st))[0]
        if st:
            compare(a, o, 1e-3 * sm.trunc, fp16_trunc=sm.trunc)
        else:
            compare(a, o, 1e-5)
    from paper_2410_21149_gb300 import _capi
    b = _capi.cvx_batch_create(1, 1)
    with pytest.raises(_capi.CovoxError):
        _capi.cvx_batch_merge_parts(b, 257)
    _capi.cvx_batch_destroy(b)


@pytest.mark.parametrize("group,wave_limit", [(1, 0), (4, 0), (2, 3)])
def test_submap_groups_do_not_change_results(mixed, group, wave_limit):
    """The queue taking the submaps in groups of one, four or two (the last
    with rounds cut into chunks of three scans): the same submaps as the
    oracle's."""
    storages = [m % 2 for m in range(len(mixed.submaps))]
    g = run_gpu_batched(mixed, storages, sets=4, submap_group=group, wave_limit=wave_limit)
    for m, (a, st) in enumerate(zip(g, storages)):
        sm = mixed.submaps[m]
        sub = sg.Workload(mixed.name, [sm], mixed.max_weight, mixed.weight_mode, mixed.dropoff,
                          mixed.min_range, mixed.max_range, mixed.scene, st)
        o = run_oracle(sub, fp16=bool(st))[0]
        if st:
            compare(a, o, 1e-3 * sm.trunc, fp16_trunc=sm.trunc)
        else:
            compare(a, o, 1e-5)
        assert a[3]["frames"] == len(sm.scans)
    from paper_2410_21149_gb300 import _capi
    b = _capi.cvx_batch_create(1, 1)
    with pytest.raises(_capi.CovoxError):
        _capi.cvx_batch_submap_group(b, -1)
    _capi.cvx_batch_destroy(b)


def test_batched_equals_per_scan_path():
    wl = sg.make_c1(n_frames=4)
    wl2 = sg.make_c3(n_scans=4, scans_per_submap=2, rows=16, cols=256, n_boxes=300)
    wl.submaps = wl.submaps + wl2.submaps     # room + two LiDAR submaps, voxel sizes differ
    gb = run_gpu_batched(wl)
    for m, sm in enumerate(wl.submaps):
        sub = sg.Workload(wl.name, [sm], wl.max_weight, wl.weight_mode, wl.dropoff, wl.min_range,
                          wl.max_range, wl.scene, 0)
        gs = run_gpu(sub)[0]
        compare(gb[m], (*sort_blocks(gs[0], gs[1], gs[2]), {}), 1e-5)


@pytest.mark.parametrize("pipelined", [False, True])
def test_batched_graph_capture_replay(mixed, pipelined):
    g = run_gpu_batched(mixed, graph=True, pipelined=pipelined)
    e = run_gpu_batched(mixed)
    for a, b in zip(g, e):
        compare(a, (*sort_blocks(b[0], b[1], b[2]), {}), 1e-3 * 0.6, fp16_trunc=0.6)


def test_batched_rejects_bad_arguments():
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    sub = cvx.Submap(0.1, 0.3)
    b = _capi.cvx_batch_create(2, 4)
    pts = torch.zeros((8, 3), device="cuda")
    T = np.eye(3, 4, dtype=np.float32)
    with pytest.raises(cvx.CovoxError):
        _capi.cvx_integrate_batch(b, [sub.handle, sub.handle], [(0, pts, T, None, cvx.integrate_params())])
    with pytest.raises(cvx.CovoxError):
        _capi.cvx_integrate_batch(b, [sub.handle], [(1, pts, T, None, cvx.integrate_params())])
    # empty scans are not frames
    _capi.cvx_integrate_batch(b, [sub.handle], [(0, torch.zeros((0, 3), device="cuda"), T, None,
                                                  cvx.integrate_params())])
    torch.cuda.synchronize()
    assert sub.counters()["frames"] == 0 and _capi.cvx_batch_error(b) == 0
    _capi.cvx_batch_destroy(b)


def test_batched_single_submap_many_frames_four_sets():
    """One submap, 12 frames in one launch (several scans of the same submap
    in flight at once), four sets against two, one and the oracle."""
    wl = sg.make_c2(n_frames=12, width=320, height=240)
    o = run_oracle(wl)[0]
    for pipelined, sets in ((True, 4), (True, 0), (False, 0)):
        g = run_gpu_batched(wl, pipelined=pipelined, sets=sets, pts_per_cta=512, local_blocks=-1)[0]
        compare(g, o, 1e-5)
        assert g[3]["frames"] == 12 and g[3]["observations"] == o[3]["obs"]



def test_reset_many_submaps_then_reintegrate(mixed):
    """cvx_reset_submaps over 6 mixed submaps after a batched launch (and over
    50 more, past one launch's 48) leaves empty submaps with zero counters, and
    integrating again gives the oracle's result, as for fresh submaps."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    from _harness import int_params
    storages = [m % 2 for m in range(len(mixed.submaps))]
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, mixed.max_weight, st, max_blocks=1 << 16, sets=4)
            for sm, st in zip(mixed.submaps, storages)]
    keep, scans = [], []
    for m, sm in enumerate(mixed.submaps):
        for sc in sm.scans:
            pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
            keep.append(pts)
            scans.append((m, pts, sc.T_sub_sensor, None, int_params(mixed, sc)))
    handles = [s.handle for s in subs]
    batch = _capi.cvx_batch_create(len(subs), len(scans))
    for rep in range(2):
        _capi.cvx_integrate_batch(batch, handles, scans)
        _capi.cvx_reset_submaps(handles)
        torch.cuda.synchronize()
        for s in subs:
            c = s.counters()
            assert s.num_blocks() == 0 and c["frames"] == 0 and c["observations"] == 0 and s.status() == 0
    _capi.cvx_integrate_batch(batch, handles, scans)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(batch) == 0
    for m, (sm, sub, st) in enumerate(zip(mixed.submaps, subs, storages)):
        keys, D, W = (t.cpu().numpy() for t in sub.extract())
        D = D.astype(np.float64) * (np.float64(np.float32(sm.trunc)) if st else 1.0)
        one = sg.Workload(mixed.name, [sm], mixed.max_weight, mixed.weight_mode, mixed.dropoff,
                          mixed.min_range, mixed.max_range, mixed.scene, st)
        o = run_oracle(one, fp16=bool(st))[0]
        g = (keys, D, W.astype(np.float64), sub.counters(), sub.status())
        if st:
            compare(g, o, 1e-3 * sm.trunc, fp16_trunc=sm.trunc)
        else:
            compare(g, o, 1e-5)
    _capi.cvx_batch_destroy(batch)
    for s in subs:
        s.close()
    # more submaps than one reset launch covers
    wl = sg.make_c1(n_frames=1)
    sm = wl.submaps[0]
    pts = torch.from_numpy(np.ascontiguousarray(sm.scans[0].points)).cuda()
    many = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, m % 2, max_blocks=1 << 10) for m in range(50)]
    for s in many:
        s.integrate(pts, sm.scans[0].T_sub_sensor, int_params(wl, sm.scans[0]))
    assert all(s.num_blocks() > 0 for s in many)
    _capi.cvx_reset_submaps([s.handle for s in many])
    assert all(s.num_blocks() == 0 and s.counters()["valid_points"] == 0 for s in many)
    s = many[49]
    s.integrate(pts, sm.scans[0].T_sub_sensor, int_params(wl, sm.scans[0]))
    keys, D, W = (t.cpu().numpy() for t in s.extract())
    o = run_oracle(sg.Workload(wl.name, [sm], wl.max_weight, wl.weight_mode, wl.dropoff, wl.min_range,
                               wl.max_range, wl.scene, 1), fp16=True)[0]
    compare((keys, D.astype(np.float64) * np.float64(np.float32(sm.trunc)), W.astype(np.float64), s.counters(),
             s.status()), o, 1e-3 * sm.trunc, fp16_trunc=sm.trunc)
    for s in many:
        s.close()
    with pytest.raises(_capi.CovoxError):
        _capi.cvx_reset_submaps([0])
