"""The no-allocation entry point against the regular one (GPU).

cvx_integrate_scan_noalloc() serves callers that cannot allocate device
memory (a real-time loop that must not allocate after start-up, a host whose
memory manager owns all device memory, a plugin barred from the allocator):
they own the submap storage and the library keeps its per-scan scratch in a
fixed device array.  Two scans in a row through it must give the same blocks,
distances and weights as two scans through cvx_integrate_scan(), within the
float32 parity tolerances of the other GPU tests.  The test allocates its
buffers with torch; the entry point itself allocates nothing.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import scenegen as sg
from _harness import int_params, sort_blocks

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
W_REL, W_FLOOR = 1e-4, 1e-6


def _view(cvx, torch, vs, trunc, max_w, max_blocks, slots):
    bufs = {
        "keys": torch.full((slots,), -1, dtype=torch.int64, device="cuda"),
        "vals": torch.full((slots,), -1, dtype=torch.int32, device="cuda"),
        "bkeys": torch.zeros((max_blocks, 3), dtype=torch.int32, device="cuda"),
        "D": torch.zeros((max_blocks, 512), dtype=torch.float32, device="cuda"),
        "W": torch.zeros((max_blocks, 512), dtype=torch.float32, device="cuda"),
        "state": torch.zeros((cvx._capi.CVX_SUBMAP_STATE_BYTES,), dtype=torch.uint8, device="cuda"),
    }
    v = cvx._capi.cvx_submap_view(bufs["keys"].data_ptr(), bufs["vals"].data_ptr(), slots,
                                  bufs["bkeys"].data_ptr(), bufs["D"].data_ptr(), bufs["W"].data_ptr(),
                                  bufs["state"].data_ptr(), max_blocks, vs, trunc, max_w)
    return v, bufs


def test_noalloc_matches_regular_entry_point_two_scans():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_21149_gb300 as cvx
    wl = sg.make_c2(n_frames=2, width=320, height=240)
    sm = wl.submaps[0]
    scans = sm.scans[:2]

    # regular entry point
    sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, cvx.CVX_STORE_F32, max_blocks=4096)
    for sc in scans:
        sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, int_params(wl, sc))
    kr, Dr, Wr = (t.cpu().numpy() for t in sub.extract())
    assert sub.status() == 0
    sub.close()

    # no-allocation entry point, two calls in a row on caller-owned storage
    view, bufs = _view(cvx, torch, sm.voxel_size, sm.trunc, wl.max_weight, 4096, 8192)
    for sc in scans:
        pts = torch.from_numpy(sc.points).cuda()
        st = cvx._capi.cvx_integrate_scan_noalloc(view, pts, sc.T_sub_sensor, None, int_params(wl, sc))
        assert st == 0, st
    torch.cuda.synchronize()
    state = bufs["state"].cpu().numpy()
    nb = int(state[:4].view(np.int32)[0])
    errs = state[12:16].view(np.int32)[0] | state[8:12].view(np.int32)[0]
    assert errs == 0
    kn = bufs["bkeys"][:nb].cpu().numpy()
    Dn = bufs["D"][:nb].cpu().numpy()
    Wn = bufs["W"][:nb].cpu().numpy()

    kr, Dr, Wr = sort_blocks(kr, Dr.astype(np.float64), Wr.astype(np.float64))
    kn, Dn, Wn = sort_blocks(kn, Dn.astype(np.float64), Wn.astype(np.float64))
    assert np.array_equal(kr, kn), "block sets differ"
    assert (np.abs(Wn - Wr) <= W_REL * np.abs(Wr) + W_FLOOR).all()
    both = (Wr > W_FLOOR) & (Wn > W_FLOOR)
    assert np.abs(Dn - Dr)[both].max() <= D_TOL
    assert both.sum() > 10000

    # and directly against the CPU oracle (the same two frames)
    from _harness import compare, run_oracle
    wl.submaps[0].scans = scans
    orc = run_oracle(wl)[0]
    compare((kn, Dn, Wn, {}, 0), orc, D_TOL)


def test_noalloc_rejects_views_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_21149_gb300 as cvx
    over = cvx._capi.CVX_NOALLOC_MAX_BLOCKS + 1
    view, bufs = _view(cvx, torch, 0.05, 0.15, 1e4, 8, 16)
    view.max_blocks = over
    pts = torch.zeros((4, 3), device="cuda")
    T = np.eye(3, 4, dtype=np.float32).reshape(12)
    st = cvx._capi.cvx_integrate_scan_noalloc(view, pts, T, None, cvx.integrate_params())
    assert st == cvx._capi.CVX_ERR_CAPACITY
