"""Shared test harness: run a workload through the CUDA library and through
the oracle, and compare the submaps element by element."""
from __future__ import annotations

import numpy as np

import scenegen as sg


def int_params(wl: sg.Workload, scan: sg.Scan, **over):
    import paper_2410_21149_gb300 as cvx
    kw = dict(weight_mode=wl.weight_mode, dropoff=wl.dropoff, min_range=wl.min_range,
              max_range=wl.max_range, sensor=scan.sensor, height=scan.height, width=scan.width)
    kw.update(over)
    return cvx.integrate_params(**kw)


def run_gpu(wl: sg.Workload, storage=None, max_blocks=1 << 17, point_weights=None, pipelined=False, colors=None,
            **over):
    """Integrate every submap of the workload; returns a list of
    (keys [nb,3] int32, D [nb,512] float64 metres, W [nb,512] float64, counters,
    status[, C [nb,3,512] float64 with colors[m][k] given])."""
    import torch
    import paper_2410_21149_gb300 as cvx
    storage = wl.storage if storage is None else storage
    out = []
    for m, sm in enumerate(wl.submaps):
        sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, storage, max_blocks=max_blocks,
                         pipelined=pipelined, color=colors is not None)
        for k, sc in enumerate(sm.scans):
            pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
            pw = None
            if point_weights is not None:
                pw = torch.from_numpy(np.ascontiguousarray(point_weights[m][k], np.float32)).cuda()
            col = None if colors is None else torch.from_numpy(np.ascontiguousarray(colors[m][k], np.float32)).cuda()
            sub.integrate(pts, sc.T_sub_sensor, int_params(wl, sc, **over), pw, colors=col)
        keys, D, W = sub.extract()
        torch.cuda.synchronize()
        keys = keys.cpu().numpy()
        D = D.cpu().numpy().astype(np.float64)
        W = W.cpu().numpy().astype(np.float64)
        if storage == 1:
            D = D * np.float64(np.float32(sm.trunc))
        res = (keys, D, W, sub.counters(), sub.status())
        if colors is not None:
            res = res + (sub.extract_colors().cpu().numpy().astype(np.float64),)
        out.append(res)
        sub.close()
    return out


def run_oracle(wl: sg.Workload, fp16=None, point_weights=None, carve=False, weight_mode=None, colors=None):
    import oracle as orc
    fp16 = bool(wl.storage) if fp16 is None else fp16
    weight_mode = wl.weight_mode if weight_mode is None else weight_mode
    out = []
    for m, sm in enumerate(wl.submaps):
        om = orc.OracleSubmap(sm.voxel_size, sm.trunc, wl.max_weight, fp16)
        tot = {}
        for k, sc in enumerate(sm.scans):
            pw = None if point_weights is None else point_weights[m][k]
            st = om.integrate(sc.points, sc.T_sub_sensor, pw, weight_mode, wl.dropoff,
                              wl.min_range, wl.max_range, sc.sensor, carve=carve,
                              colors=None if colors is None else colors[m][k])
            for key, v in st.items():
                tot[key] = tot.get(key, 0) + v
        keys, D, W = om.extract()
        res = (keys, D, W, tot)
        if colors is not None:
            res = res + (om.extract_colors(),)
        out.append(res)
    return out


def sort_blocks(keys, D, W):
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    return keys[order], D[order], W[order]


def compare(gpu, orc, d_tol, w_rel=1e-4, w_floor=1e-6, fp16_trunc=None, d_tol_w=0.0):
    """Block sets bit-exact; W within w_rel relative (abs floor w_floor, or one
    half ulp for FP16 storage); D within d_tol + d_tol_w / W where both
    weights are above the floor (d_tol_w: the spread of a voxel's distances,
    2 trunc, times an absolute error of its weights, which moves the weighted
    mean by at most that over W).  Returns a dict of the largest errors."""
    kg, Dg, Wg, cnt, status = gpu[:5]
    ko, Do, Wo, tot = orc[:4]
    assert status == 0, status
    kg, Dg, Wg = sort_blocks(kg, Dg, Wg)
    assert kg.shape == ko.shape, (kg.shape, ko.shape)
    assert np.array_equal(kg, ko), "block sets differ"
    if fp16_trunc is None:
        wtol = w_rel * np.abs(Wo) + w_floor
    else:
        ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(Wo), 2.0 ** -14))) - 10)
        wtol = ulp + w_floor
    werr = np.abs(Wg - Wo)
    assert (werr <= wtol).all(), f"W error {werr.max()} (at W={Wo.flat[np.argmax(werr - wtol)]})"
    both = (Wo > w_floor) & (Wg > w_floor)
    same = ((Wo > 0) == (Wg > 0)) | (np.maximum(Wo, Wg) <= 10 * w_floor)
    assert same.all(), "voxel sets with weight differ"
    derr = np.abs(Dg - Do)[both]
    dtol = d_tol + d_tol_w / np.maximum(Wo[both], 1e-30)
    assert derr.size == 0 or (derr <= dtol).all(), f"D error {derr.max()}"
    return {"d_max": float(derr.max()) if derr.size else 0.0, "w_max": float(werr.max()),
            "voxels": int(both.sum()), "blocks": int(len(ko))}


def compare_colors(gpu, orc, c_tol, w_floor=1e-6, c_tol_w=0.0):
    """Fused colours of the voxels whose weights are above the floor on both
    sides within c_tol + c_tol_w / W (c_tol_w: the colour range times an
    absolute error of the voxel's weights); zero colour where the oracle's
    weight is zero.  Returns the largest error."""
    kg, Wg, Cg = gpu[0], gpu[2], gpu[5]
    ko, Wo, Co = orc[0], orc[2], orc[4]
    order = np.lexsort((kg[:, 2], kg[:, 1], kg[:, 0]))
    kg, Wg, Cg = kg[order], Wg[order], Cg[order]
    assert np.array_equal(kg, ko), "block sets differ"
    both = (Wo > w_floor) & (Wg > w_floor)
    err = np.abs(Cg - Co).max(axis=1)[both]
    tol = c_tol + c_tol_w / np.maximum(Wo[both], 1e-30)
    assert err.size == 0 or (err <= tol).all(), f"C error {err.max()}"
    assert (Cg.max(axis=1)[(Wo == 0) & (Wg == 0)] == 0).all(), "colour where nothing was observed"
    return float(err.max()) if err.size else 0.0


def run_gpu_batched(wl: sg.Workload, storages=None, max_blocks=1 << 16, graph=False, pipelined=False,
                    wave_limit=0, point_weights=None, sets=0, colors=None, merge_parts=0, submap_group=0, **over):
    """Integrate all submaps of the workload with one cvx_integrate_batch call
    (scans of a submap are frames in order).  Returns the run_gpu tuple list."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    storages = storages or [wl.storage] * len(wl.submaps)
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, st, max_blocks=max_blocks, pipelined=pipelined,
                       sets=sets, color=colors is not None) for sm, st in zip(wl.submaps, storages)]
    keep = []
    scans = []
    # interleave submaps' scans (any order works; frames keep per-submap order)
    k = 0
    while any(k < len(sm.scans) for sm in wl.submaps):
        for m, sm in enumerate(wl.submaps):
            if k < len(sm.scans):
                sc = sm.scans[k]
                pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
                keep.append(pts)
                pw = None
                if point_weights is not None:
                    pw = torch.from_numpy(np.ascontiguousarray(point_weights[m][k], np.float32)).cuda()
                    keep.append(pw)
                desc = (m, pts, sc.T_sub_sensor, pw, int_params(wl, sc, **over))
                if colors is not None:
                    col = torch.from_numpy(np.ascontiguousarray(colors[m][k], np.float32)).cuda()
                    keep.append(col)
                    desc = desc + (col,)
                scans.append(desc)
        k += 1
    batch = _capi.cvx_batch_create(len(subs), len(scans))
    _capi.cvx_batch_wave_limit(batch, wave_limit)
    _capi.cvx_batch_merge_parts(batch, merge_parts)
    _capi.cvx_batch_submap_group(batch, submap_group)
    handles = [s.handle for s in subs]
    if graph:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            _capi.cvx_integrate_batch(batch, handles, scans, s)
        for sub in subs:
            sub.reset()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
    else:
        _capi.cvx_integrate_batch(batch, handles, scans)
    torch.cuda.synchronize()
    err = _capi.cvx_batch_error(batch)
    out = []
    for sm, sub, st in zip(wl.submaps, subs, storages):
        keys, D, W = sub.extract()
        keys = keys.cpu().numpy()
        D = D.cpu().numpy().astype(np.float64)
        W = W.cpu().numpy().astype(np.float64)
        if st == 1:
            D = D * np.float64(np.float32(sm.trunc))
        res = (keys, D, W, sub.counters(), sub.status() or err)
        if colors is not None:
            res = res + (sub.extract_colors().cpu().numpy().astype(np.float64),)
        out.append(res)
        sub.close()
    _capi.cvx_batch_destroy(batch)
    return out
