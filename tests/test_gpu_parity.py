"""GPU parity: the CUDA library against the CPU oracle, element by element.

Tolerances: block sets bit-exact; D within 1e-5 m (float32 storage) or
1e-3 trunc (float16 storage, against the oracle's float16 storage mode); W
within 1e-4 relative with a 1e-6 absolute floor (float32) or one half ulp
(float16).  Cases span several CTA tiles with ragged tails, the empty scan,
invalid points, negative coordinates and the error paths.
"""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

D_TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_21149_gb300 as cvx
    cvx._capi.lib()


def test_library_is_in_tree():
    import os
    import paper_2410_21149_gb300 as cvx
    L = cvx._capi.lib()
    assert os.path.samefile(L._name, cvx._capi.LIB_PATH)


def test_room_10_frames_fp32():
    wl = sg.make_c1()
    g = run_gpu(wl)
    o = run_oracle(wl)
    r = compare(g[0], o[0], D_TOL_F32)
    cnt, tot = g[0][3], o[0][3]
    assert cnt["valid_points"] == tot["valid"]
    assert cnt["observations"] == tot["obs"]
    assert cnt["blocks_touched"] == tot["blocks"]
    assert cnt["voxels_merged"] <= tot["voxels"]
    assert r["voxels"] > 30000


@pytest.mark.parametrize("dropoff", [0, 1, 2])
def test_multiroom_quadratic_dropoff_fp32(dropoff):
    wl = sg.make_c2(n_frames=3, dropoff=dropoff)
    compare(run_gpu(wl)[0], run_oracle(wl)[0], D_TOL_F32)


def test_multiroom_fp16_storage():
    wl = sg.make_c2(n_frames=4, storage=1)
    tr = wl.submaps[0].trunc
    compare(run_gpu(wl)[0], run_oracle(wl, fp16=True)[0], 1e-3 * tr, fp16_trunc=tr)


def test_multiroom_fp16_error_vs_fp64():
    """Stated error of FP16 storage against the unrounded FP64 oracle."""
    wl = sg.make_c2(n_frames=4, storage=1)
    g = run_gpu(wl)[0]
    o = run_oracle(wl, fp16=False)[0]
    from _harness import sort_blocks
    kg, Dg, Wg = sort_blocks(g[0], g[1], g[2])
    ko, Do, Wo, _ = o
    assert np.array_equal(kg, ko)
    m = Wo > 1e-6
    err = np.abs(Dg - Do)[m]
    # a few half ulps of the normalised distance, times trunc
    assert err.max() < 8 * 2.0 ** -11 * wl.submaps[0].trunc


def test_lidar_submaps_fp32():
    wl = sg.make_c3(n_scans=6, scans_per_submap=3, n_boxes=400)
    g = run_gpu(wl)
    o = run_oracle(wl)
    for a, b in zip(g, o):
        compare(a, b, D_TOL_F32)


@pytest.mark.parametrize("ppc", [256, 700, 2048])
def test_tile_sizes_and_ragged_tail(ppc):
    wl = sg.make_c1(n_frames=3)
    for s in wl.submaps[0].scans:
        s.points = s.points[: 19200 - 37]   # not a multiple of any tile
    compare(run_gpu(wl, pts_per_cta=ppc)[0], run_oracle(wl)[0], D_TOL_F32)


def test_point_order_invariance():
    wl = sg.make_c1(n_frames=3)
    rng = np.random.default_rng(5)
    g1 = run_gpu(wl)[0]
    for s in wl.submaps[0].scans:
        s.points = s.points[rng.permutation(len(s.points))]
    g2 = run_gpu(wl)[0]
    o = run_oracle(wl)[0]
    compare(g1, o, D_TOL_F32)
    compare(g2, o, D_TOL_F32)


def test_empty_nan_and_single_point_scans():
    import torch
    import paper_2410_21149_gb300 as cvx
    sub = cvx.Submap(0.1, 0.3)
    T = np.array([1, 0, 0, 0.05, 0, 1, 0, -3.2, 0, 0, 1, 0.7], np.float32)
    p = cvx.integrate_params()
    sub.integrate(torch.empty((0, 3), device="cuda"), T, p)
    sub.integrate(torch.full((1000, 3), float("nan"), device="cuda"), T, p)
    one = np.array([[0.3, -0.4, 2.0]], np.float32)
    sub.integrate(torch.from_numpy(one).cuda(), T, p)
    keys, D, W = sub.extract()
    import oracle as orc
    om = orc.OracleSubmap(0.1, 0.3)
    om.integrate(one, T)
    ko, Do, Wo = om.extract()
    from _harness import sort_blocks
    kg, Dg, Wg = sort_blocks(keys.cpu().numpy(), D.cpu().double().numpy(), W.cpu().double().numpy())
    assert np.array_equal(kg, ko)
    assert np.abs(Dg - Do).max() < D_TOL_F32 and np.array_equal(Wg, Wo)
    assert (ko < 0).any()              # negative block coordinates exercised
    c = sub.counters()
    assert c["valid_points"] == 1 and c["frames"] == 2


def test_capacity_error_leaves_voxels_unchanged():
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c1(n_frames=2)
    sub = cvx.Submap(0.1, 0.3, max_blocks=8, hash_slots=16)
    s = wl.submaps[0].scans[0]
    sub.integrate(torch.from_numpy(s.points).cuda(), s.T_sub_sensor, cvx.integrate_params())
    assert sub.status() == cvx._capi.CVX_ERR_CAPACITY
    keys, D, W = sub.extract()
    assert len(keys) == 8 and float(W.abs().max()) == 0.0 and float(D.abs().max()) == 0.0


def test_key_range_error():
    import torch
    import paper_2410_21149_gb300 as cvx
    sub = cvx.Submap(0.1, 0.3)
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    pts = torch.tensor([[0.0, 0.0, 2.0], [0.0, 0.0, 2.0e6]], device="cuda")
    sub.integrate(pts, T, cvx.integrate_params(max_range=1e9))
    assert sub.status() == cvx._capi.CVX_ERR_KEY_RANGE
    keys, D, W = sub.extract()
    assert float(W.abs().max()) == 0.0   # the scan's merge was skipped


def test_invalid_arguments_are_synchronous():
    import torch
    import paper_2410_21149_gb300 as cvx
    sub = cvx.Submap(0.1, 0.3)
    pts = torch.zeros((4, 3), device="cuda")
    bad_T = np.full(12, np.nan, np.float32)
    with pytest.raises(cvx.CovoxError) as e:
        sub.integrate(pts, bad_T, cvx.integrate_params())
    assert e.value.status == cvx._capi.CVX_ERR_INVALID_ARG
    T = np.eye(3, 4, dtype=np.float32)
    with pytest.raises(cvx.CovoxError):
        sub.integrate(pts, T, cvx.integrate_params(weight_mode=2))   # no per-point weights
    sub2 = cvx.Submap(0.1, 0.1)
    with pytest.raises(cvx.CovoxError):
        sub2.integrate(pts, T, cvx.integrate_params(dropoff=1))      # trunc must exceed vs
    with pytest.raises(cvx.CovoxError):
        cvx.Submap(0.1, 0.3, hash_slots=1000)                        # not a power of two


def test_cudamalloc_path_and_reset():
    import torch
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c1(n_frames=2)
    sub = cvx.Submap(0.1, 0.3, use_torch_allocator=False)
    p = cvx.integrate_params()
    for s in wl.submaps[0].scans:
        sub.integrate(torch.from_numpy(s.points).cuda(), s.T_sub_sensor, p)
    k1 = sub.extract()[0].cpu().numpy()
    sub.reset()
    assert sub.num_blocks() == 0
    for s in wl.submaps[0].scans:
        sub.integrate(torch.from_numpy(s.points).cuda(), s.T_sub_sensor, p)
    g = list(x.cpu().numpy().astype(np.float64) if i else x.cpu().numpy()
             for i, x in enumerate(sub.extract()))
    assert sorted(map(tuple, k1)) == sorted(map(tuple, g[0]))
    compare((g[0], g[1], g[2], None, 0), run_oracle(wl)[0], D_TOL_F32)


@pytest.mark.parametrize("ppc,lb", [(256, 16), (1024, 2), (2048, 16), (512, 1)])
def test_organised_tiles_and_local_slot_overflow(ppc, lb):
    """Organised tiling at several tile heights; few shared-memory block slots
    force the direct global-accumulation path."""
    wl = sg.make_c2(n_frames=2, width=320, height=240)
    compare(run_gpu(wl, pts_per_cta=ppc, local_blocks=lb)[0], run_oracle(wl)[0], D_TOL_F32)


def test_global_accumulation_mode_lidar():
    """local_blocks = -1: every observation goes straight to the global sums."""
    wl = sg.make_c3(n_scans=4, scans_per_submap=4, n_boxes=300)
    compare(run_gpu(wl, local_blocks=-1)[0], run_oracle(wl)[0], D_TOL_F32)
