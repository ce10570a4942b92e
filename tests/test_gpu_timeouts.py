"""The bounded waits of the kernels run out and report, without faulting or
hanging the GPU, and the library recovers in the same process (GPU).

- Grid barriers of the batched persistent kernel: a test hook makes one CTA
  leave before its first arrival and shortens the poll limit; the other CTAs
  give up, cvx_batch_error() reports CVX_ERR_TIMEOUT.  After a reset (which
  also drops the per-scan sums the aborted launch left unmerged) the same
  batch object and submaps integrate normally and match the oracle.
- Publication of a block's pool index: a caller-owned hash (the
  allocation-free entry point's view) whose slots hold the block's key with
  the pool index never published; the activating thread waits out its poll
  limit, the scan records CVX_ERR_TIMEOUT in the state's error words and its
  merge is skipped; a fresh view then integrates the same scan normally.
"""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, int_params, run_oracle, sort_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_grid_barrier_timeout_then_recovery():
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    wl = sg.make_c1(n_frames=2)
    wl2 = sg.make_c3(n_scans=4, scans_per_submap=2, rows=16, cols=256, n_boxes=300)
    wl.submaps = wl.submaps + wl2.submaps
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, 0, max_blocks=1 << 14) for sm in wl.submaps]
    keep, scans = [], []
    for m, sm in enumerate(wl.submaps):
        for sc in sm.scans:
            p = torch.from_numpy(sc.points).cuda()
            keep.append(p)
            scans.append((m, p, sc.T_sub_sensor, None, int_params(wl, sc)))
    b = _capi.cvx_batch_create(len(subs), len(scans))
    handles = [s.handle for s in subs]
    _capi.cvx_batch_test_missing_cta(b, 1, 20000)
    _capi.cvx_integrate_batch(b, handles, scans)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(b) == _capi.CVX_ERR_TIMEOUT
    # recovery: hook off, reset, the same batch again
    _capi.cvx_batch_test_missing_cta(b, -1, 0)
    for s in subs:
        s.reset()
    _capi.cvx_integrate_batch(b, handles, scans)
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(b) == 0
    for m, (sm, sub) in enumerate(zip(wl.submaps, subs)):
        keys, D, W = (t.cpu().numpy() for t in sub.extract())
        g = (keys, D.astype(np.float64), W.astype(np.float64), sub.counters(), sub.status())
        one = sg.Workload(wl.name, [sm], wl.max_weight, wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range,
                          wl.scene, 0)
        compare(g, run_oracle(one)[0], 1e-5)
        assert g[3]["frames"] == len(sm.scans)
    _capi.cvx_batch_destroy(b)
    for s in subs:
        s.close()


def _pack_key(b):
    return ((int(b[0]) + (1 << 20)) << 42) | ((int(b[1]) + (1 << 20)) << 21) | (int(b[2]) + (1 << 20))


def test_unpublished_block_times_out_then_recovers():
    import torch
    import oracle as orc
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    vs, tr, slots, nb = 0.1, 0.3, 64, 64
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    p = np.array([[0.4, 0.4, 4.4]], np.float32)        # its band lies in block (0, 0, 5)
    vox, _, _, _ = orc.point_obs(p[0], T, vs, tr)
    blocks = np.unique(np.floor_divide(vox, 8), axis=0)
    assert blocks.tolist() == [[0, 0, 5]]
    prm = cvx.integrate_params()

    def view(poison):
        key = _pack_key(blocks[0])
        keys = torch.full((slots,), key if poison else -1, dtype=torch.int64, device="cuda")
        bufs = {"keys": keys, "vals": torch.full((slots,), -1, dtype=torch.int32, device="cuda"),
                "bkeys": torch.zeros((nb, 3), dtype=torch.int32, device="cuda"),
                "D": torch.zeros((nb, 512), dtype=torch.float32, device="cuda"),
                "W": torch.zeros((nb, 512), dtype=torch.float32, device="cuda"),
                "state": torch.zeros((_capi.CVX_SUBMAP_STATE_BYTES,), dtype=torch.uint8, device="cuda")}
        v = _capi.cvx_submap_view(bufs["keys"].data_ptr(), bufs["vals"].data_ptr(), slots, bufs["bkeys"].data_ptr(),
                                  bufs["D"].data_ptr(), bufs["W"].data_ptr(), bufs["state"].data_ptr(), nb, vs, tr,
                                  1e4)
        return v, bufs

    pts = torch.from_numpy(p).cuda()
    v, bufs = view(poison=True)
    assert _capi.cvx_integrate_scan_noalloc(v, pts, T, None, prm) == 0
    torch.cuda.synchronize()
    st = bufs["state"].cpu().numpy()
    sticky = int(st[12:16].view(np.int32)[0])
    assert sticky & 4, sticky                       # CVX_ERR_TIMEOUT bit of the sticky word
    assert float(bufs["W"].abs().sum()) == 0.0      # the scan's merge was skipped
    # a fresh view integrates the same scan normally
    v, bufs = view(poison=False)
    assert _capi.cvx_integrate_scan_noalloc(v, pts, T, None, prm) == 0
    torch.cuda.synchronize()
    st = bufs["state"].cpu().numpy()
    assert int(st[12:16].view(np.int32)[0]) == 0
    n = int(st[:4].view(np.int32)[0])
    om = orc.OracleSubmap(vs, tr, 1e4)
    om.integrate(p, T)
    ko, Do, Wo = om.extract()
    kg, Dg, Wg = sort_blocks(bufs["bkeys"][:n].cpu().numpy(), bufs["D"][:n].cpu().double().numpy(),
                             bufs["W"][:n].cpu().double().numpy())
    compare((kg, Dg, Wg, {}, 0), (ko, Do, Wo, {}), 1e-5)
