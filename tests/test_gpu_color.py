"""GPU parity of colour integration ("TSDF + Color", coVoxSLAM Sec. IV) against
the CPU oracle, element by element.

Every observation carries its point's colour with the observation's weight;
each voxel's colour follows the weighted running mean of the distance,
C <- (C W + S_wc) / (W + S_w).  Colours are a seeded procedural albedo of the
surface point (scenegen.point_colors).  Cases: the room workload on the
per-scan path and on the pipelined per-scan path; a 640x480 multiroom prefix
with the quadratic weight and behind-surface drop-off, in FP32 and FP16
storage; the batched launch over submaps of both sensor kinds with one, two
and four per-scan sets; non-finite colours, which drop their points; reset;
the argument checks.

Tolerances: blocks bit-exact, D and W as in the plain parity tests, colour
C_TOL = 3e-5 absolute for colours in [0, 1]: the colour sums are the same
FP32 sums as the distance sums, whose 1e-5 m tolerance over the 0.3 m range
of D - trunc is a relative 3.3e-5; drop-off runs add floor / W (the weights'
FP32 error floor times the colour range 1, as the distance test adds
2 trunc floor / W).
"""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, compare_colors, run_gpu, run_gpu_batched, run_oracle

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
C_TOL = 3e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _colors(wl, seed=0):
    return [[sg.point_colors(sc, seed) for sc in sm.scans] for sm in wl.submaps]


def _floor(wl, w0_max, d_err=1e-6):
    sm = wl.submaps[0]
    return 1e-6 if wl.dropoff == 0 else max(1e-6, w0_max * d_err / (sm.trunc - sm.voxel_size))


@pytest.mark.parametrize("pipelined", [False, True])
def test_room_colours(pipelined):
    wl = sg.make_c1(n_frames=4)
    cols = _colors(wl)
    g = run_gpu(wl, colors=cols, pipelined=pipelined)[0]
    o = run_oracle(wl, colors=cols)[0]
    r = compare(g, o, D_TOL)
    e = compare_colors(g, o, C_TOL)
    assert r["voxels"] > 5000
    assert g[3]["valid_points"] == o[3]["valid"] and g[3]["observations"] == o[3]["obs"]
    assert e < C_TOL


@pytest.mark.parametrize("storage", [0, 1])
def test_multiroom_colours_with_dropoff(storage):
    wl = sg.make_c2(n_frames=3, storage=storage)
    cols = _colors(wl, 1)
    g = run_gpu(wl, colors=cols)[0]
    o = run_oracle(wl, colors=cols)[0]
    # the largest base weight 1/z^2 of the scans (z >= min_range 0.1 m)
    zmin = min(float(np.nanmin(sc.points[:, 2][sc.points[:, 2] > 0])) for sc in wl.submaps[0].scans)
    fl = _floor(wl, 1.0 / max(zmin, wl.min_range) ** 2)
    if storage == 0:
        compare(g, o, D_TOL, w_floor=fl, d_tol_w=2 * wl.submaps[0].trunc * fl)
    else:
        compare(g, o, 1e-3 * wl.submaps[0].trunc, fp16_trunc=wl.submaps[0].trunc, w_floor=fl,
                d_tol_w=2 * wl.submaps[0].trunc * fl)
    # FP16 storage: colours are FP32 in both modes, but the stored W they use is the
    # half-rounded one on both sides
    compare_colors(g, o, C_TOL, w_floor=fl, c_tol_w=fl)


@pytest.mark.parametrize("sets", [0, 2, 4])
def test_batched_colours(sets):
    wl = sg.make_c1(n_frames=3)
    wl2 = sg.make_c3(n_scans=6, scans_per_submap=3, rows=16, cols=256, n_boxes=300)
    wl.submaps = wl.submaps + wl2.submaps
    cols = _colors(wl, 2)
    g = run_gpu_batched(wl, colors=cols, sets=sets)
    for m, sm in enumerate(wl.submaps):
        one = sg.Workload(wl.name, [sm], wl.max_weight, wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range,
                          wl.scene, 0)
        o = run_oracle(one, colors=[cols[m]])[0]
        compare(g[m], o, D_TOL)
        compare_colors(g[m], o, C_TOL)
        assert g[m][3]["frames"] == len(sm.scans)


def test_non_finite_colours_drop_their_points():
    wl = sg.make_c1(n_frames=3)
    cols = _colors(wl, 3)
    rng = np.random.default_rng(14)
    for c in cols[0]:
        b = rng.choice(len(c), len(c) // 8, replace=False)
        c[b[0::3], 0] = np.nan
        c[b[1::3], 1] = np.inf
        c[b[2::3], 2] = -np.inf
    g = run_gpu(wl, colors=cols)[0]
    o = run_oracle(wl, colors=cols)[0]
    compare(g, o, D_TOL)
    compare_colors(g, o, C_TOL)
    assert g[3]["valid_points"] == o[3]["valid"] and g[3]["observations"] == o[3]["obs"]


def test_reset_clears_colours_and_argument_checks():
    import torch
    import paper_2410_21149_gb300 as cvx
    from _harness import int_params
    wl = sg.make_c1(n_frames=2)
    sm = wl.submaps[0]
    cols = _colors(wl, 4)
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, 0, max_blocks=1 << 14, color=True)
    plain = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, 0, max_blocks=1 << 14)
    sc = sm.scans[0]
    pts = torch.from_numpy(sc.points).cuda()
    col = torch.from_numpy(cols[0][0]).cuda()
    prm = int_params(wl, sc)
    with pytest.raises(cvx.CovoxError):
        sub.integrate(pts, sc.T_sub_sensor, prm)                 # a colour submap needs colours
    with pytest.raises(cvx.CovoxError):
        plain.integrate(pts, sc.T_sub_sensor, prm, colors=col)   # and only a colour submap takes them
    with pytest.raises(cvx.CovoxError):
        plain.extract_colors()
    sub.integrate(pts, sc.T_sub_sensor, prm, colors=col)
    assert float(sub.extract_colors().abs().sum()) > 0
    sub.reset()
    assert sub.num_blocks() == 0
    # after the reset the submap integrates the second scan as if new
    sc2 = sm.scans[1]
    sub.integrate(torch.from_numpy(sc2.points).cuda(), sc2.T_sub_sensor, int_params(wl, sc2),
                  colors=torch.from_numpy(cols[0][1]).cuda())
    keys, D, W = sub.extract()
    g = (keys.cpu().numpy(), D.cpu().double().numpy(), W.cpu().double().numpy(), sub.counters(), sub.status(),
         sub.extract_colors().cpu().double().numpy())
    one = sg.Workload(wl.name, [sg.SubmapWork([sc2], sm.T_world_sub, sm.voxel_size, sm.trunc)], wl.max_weight,
                      wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range, wl.scene, 0)
    o = run_oracle(one, colors=[[cols[0][1]]])[0]
    compare(g, o, D_TOL)
    compare_colors(g, o, C_TOL)
    sub.close()
    plain.close()
