#!/usr/bin/env python
"""TSDF integration throughput on GB300 (points/s, voxel-updates/s, SDF RMSE).

Default workload: plain FP32 integration of 200 pinhole frames of 640x480
(307,200 points each) on a random walk through a 30 x 30 x 5 m multi-room
building (axial noise 0.0012 z^2, 2% dropout, voxel 0.05 m, trunc 0.15 m,
quadratic weight with linear behind-surface drop-off), beside the same
workload with FP16 storage.  One step = clear the submap + integrate all 200
frames, replayed from a CUDA graph; inputs (737 MB of points) are resident in
HBM and exceed L2.  `--workload lidar` runs the LiDAR/MAV workload through
the batched path instead.

`--impl reference` times the CPU oracle (FP64, single thread) on a bounded
sample of the same workload: the only other place this file runs oracle code.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
KERNEL_SOURCES = ("paper_2410_21149_gb300/csrc/covox_dev.cuh", "paper_2410_21149_gb300/csrc/integrate_dev.cuh",
                  "paper_2410_21149_gb300/csrc/integrate.cu", "paper_2410_21149_gb300/csrc/batched.cu")


def kernel_traffic(name: str, ppc: int = 0, lb: int = 0, workload: str = ""):
    """DRAM bytes per launch from the committed ncu summary for this kernel,
    workload and launch shape, or None if there is none or the kernel sources
    changed since it was captured."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    name = f"{name}|{workload}|{ppc},{lb}"
    if name not in t:
        return None
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return t[name]["dram_bytes_per_launch"] if h.hexdigest() == t[name].get("csrc_sha256") else None


# ---------------------------------------------------------------- helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup(backend: str = "nccl"):
    """One process per GPU (torchrun environment).  The only collectives are
    the timing barrier and the reductions of the reported numbers: the
    submaps of different ranks are independent, so the data path has none."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def _coll_device():
    import torch.distributed as dist
    return "cpu" if dist.get_backend() == "gloo" else "cuda"


def barrier(ws):
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(x: float, ws: int) -> float:
    """Step time of the slowest rank."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_coll_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int) -> float:
    """Units processed by all ranks together."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_coll_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -------------------------------------------------------------- workloads
def make_workload(name: str, frames: int):
    import scenegen as sg
    if name == "multiroom":
        return sg.make_c2(n_frames=frames)
    if name == "room":
        return sg.make_c1()
    raise SystemExit(f"unknown workload {name}")


def sdf_rmse(scene, keys, D, W, vs, trunc):
    """RMSE of stored D against the analytic scene distance (clamped to +-trunc)
    over voxels with W > 0 and |D| < trunc."""
    b, l = np.nonzero((W > 0) & (np.abs(D) < trunc))
    if len(b) == 0:
        return None
    v = keys[b].astype(np.int64) * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)
    c = (v + 0.5) * np.float64(np.float32(vs))
    sdf = scene.sdf(c, trunc)
    return float(np.sqrt(np.mean((D[b, l] - sdf) ** 2)))


def multi_rmse(wl, subs, storage):
    """SDF RMSE over all submaps (voxel centres moved to the world frame)."""
    errs = []
    for sm, sub in zip(wl.submaps, subs):
        keys, D, W = (t.cpu().numpy() for t in sub.extract())
        D = D.astype(np.float64)
        if storage == 1:
            D = D * np.float64(np.float32(sm.trunc))
        W = W.astype(np.float64)
        b, l = np.nonzero((W > 0) & (np.abs(D) < sm.trunc))
        if len(b) == 0:
            continue
        v = keys[b].astype(np.int64) * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], 1)
        c = (v + 0.5) * np.float64(np.float32(sm.voxel_size)) + sm.T_world_sub[:, 3]
        sdf = (sm.scene or wl.scene).sdf(c, sm.trunc)
        errs.append((D[b, l] - sdf) ** 2)
    return float(np.sqrt(np.mean(np.concatenate(errs)))) if errs else None


def bench_multi(wl, storage, steps, warmup, ws, max_blocks=1 << 16, sequential=True, tune_force=False,
                pipelined=True, sets=4):
    """Many submaps: one batched persistent launch per step (autotuned tile
    shape, CUDA graph), beside the same scans through the per-scan path."""
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi, autotune
    stream = torch.cuda.Stream()
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, storage, max_blocks=max_blocks,
                       pipelined=pipelined, sets=sets) for sm in wl.submaps]
    handles = [s.handle for s in subs]
    # every scan's points in one device buffer (views per scan) with a pinned
    # host copy for the end-to-end timing
    scans_all = [(m, sc) for m, sm in enumerate(wl.submaps) for sc in sm.scans]
    n_points = sum(int(sc.points.shape[0]) for _, sc in scans_all)
    host_all = torch.empty((n_points, 3), dtype=torch.float32).pin_memory()
    dev_all = torch.empty((n_points, 3), dtype=torch.float32, device="cuda")
    items, o = [], 0
    for m, sc in scans_all:
        n = int(sc.points.shape[0])
        host_all[o:o + n] = torch.from_numpy(np.ascontiguousarray(sc.points))
        items.append((m, dev_all[o:o + n], sc.T_sub_sensor, sc))
        o += n
    dev_all.copy_(host_all)

    def prm(sc, ppc=0, lb=0):
        return cvx.integrate_params(wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range, sc.sensor,
                                    sc.height, sc.width, ppc, lb)

    def reset(st=None):
        _capi.cvx_reset_submaps(handles, st)

    tuned = autotune.tune_batch(handles, [(m, p, T, None, prm(sc)) for m, p, T, sc in items],
                                f"{wl.name}|st{storage}|p{int(pipelined)}|s{sets}", reset=reset, force=tune_force)
    ppc, lb = tuned["pts_per_cta"], tuned["local_blocks"]
    bscans = [(m, p, T, None, prm(sc, ppc, lb)) for m, p, T, sc in items]
    batch = _capi.cvx_batch_create(len(subs), len(bscans))

    def step_batched():
        reset(stream)
        _capi.cvx_integrate_batch(batch, handles, bscans, stream)

    def step_seq():
        reset(stream)
        for m, p, T, sc in items:
            subs[m].integrate(p, T, prm(sc, ppc, lb), None, stream)
        for s in subs:
            s.flush(stream)      # pipelined submaps: each one's last scan

    def graph_time(step):
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                g.replay()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                g.replay()
            e1.record(stream)
            barrier(ws)
        return max_over_ranks(e0.elapsed_time(e1), ws) / steps

    ms_b = graph_time(step_batched)
    # one eager step: counters, kernel time, per-wave phase times, status
    _capi.cvx_profile_start(1 << 20)
    _capi.cvx_batch_timing(batch, True)
    l0 = _capi.cvx_launch_count()
    step_batched()
    torch.cuda.synchronize()
    launches = _capi.cvx_launch_count() - l0
    _capi.cvx_profile_stop()
    _capi.cvx_batch_timing(batch, False)
    prof = _capi.cvx_profile_read()
    phases = _capi.cvx_batch_phase_times(batch)
    assert _capi.cvx_batch_error(batch) == 0 and all(s.status() == 0 for s in subs)
    cnt = [s.counters() for s in subs]
    tot = {k: sum(c[k] for c in cnt) for k in cnt[0]}
    rmse = multi_rmse(wl, subs, storage)
    ms_s = graph_time(step_seq) if sequential else None

    # end to end through the public API: the scans' points copied from pinned
    # host memory in four chunks of consecutive frame ranks (host buffer in
    # rank-major order, one copy per chunk on a side stream), each chunk's
    # batched launch starting as its copy lands while the next chunk copies,
    # every submap's counters read back.  The copies and launches of a step
    # are captured once as a CUDA graph and replayed.
    rank, per_map = [], {}
    for m, _, _, _ in items:
        rank.append(per_map.get(m, 0))
        per_map[m] = rank[-1] + 1
    rm_order = sorted(range(len(items)), key=lambda i: (rank[i], items[i][0]))
    host_rm = torch.empty((n_points, 3), dtype=torch.float32).pin_memory()
    dev_rm = torch.empty((n_points, 3), dtype=torch.float32, device="cuda")
    n_ranks = max(rank) + 1
    n_chunks = min(4, n_ranks)
    chunks, o = [], 0   # (first point, end point, scans) per chunk
    for c in range(n_chunks):
        r0, r1 = c * n_ranks // n_chunks, (c + 1) * n_ranks // n_chunks
        o0, sc_c = o, []
        for i in rm_order:
            if r0 <= rank[i] < r1:
                m, p, T, sc = items[i]
                n = int(p.shape[0])
                host_rm[o:o + n] = torch.from_numpy(np.ascontiguousarray(sc.points))
                sc_c.append((m, dev_rm[o:o + n], T, None, prm(sc, ppc, lb)))
                o += n
        chunks.append((o0, o, sc_c))
    chunk_batches = [_capi.cvx_batch_create(len(subs), max(len(c[2]), 1)) for c in chunks]
    copy_stream = torch.cuda.Stream()
    ev_copied = [torch.cuda.Event() for _ in chunks]
    ev_start = torch.cuda.Event()

    def e2e_body():
        reset(stream)
        ev_start.record(stream)
        copy_stream.wait_event(ev_start)   # the previous step no longer reads dev_rm
        with torch.cuda.stream(copy_stream):
            for c, (o0, o1, _) in enumerate(chunks):
                dev_rm[o0:o1].copy_(host_rm[o0:o1], non_blocking=True)
                ev_copied[c].record(copy_stream)
        for c, (_, _, sc_c) in enumerate(chunks):
            stream.wait_event(ev_copied[c])
            if sc_c:
                _capi.cvx_integrate_batch(chunk_batches[c], handles, sc_c, stream)

    for _ in range(warmup):
        e2e_body()
    torch.cuda.synchronize()
    g_e2e = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_e2e, stream=stream):
        e2e_body()
    torch.cuda.synchronize()

    def e2e_step():
        with torch.cuda.stream(stream):
            g_e2e.replay()
        return [s.counters() for s in subs]

    for _ in range(warmup):
        e2e_step()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(steps):
        ce = e2e_step()
    barrier(ws)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, ws) / steps
    assert sum(c["valid_points"] for c in ce) == tot["valid_points"] and all(s.status() == 0 for s in subs)
    for cb in chunk_batches:
        assert _capi.cvx_batch_error(cb) == 0
        _capi.cvx_batch_destroy(cb)
    kern_ms = prof["batched_kernel"][0] / max(prof["batched_kernel"][1], 1)
    S = 8 if storage == 0 else 4
    kbytes = 12 * n_points + 2 * S * tot["voxels_merged"] + 16 * tot["blocks_touched"]
    _capi.cvx_batch_destroy(batch)
    for s in subs:
        s.close()
    return {"ms_per_step": ms_b, "ms_per_step_per_scan_path": ms_s, "points": tot["valid_points"],
            "input_points": n_points, "observations": tot["observations"], "voxels_merged": tot["voxels_merged"],
            "blocks_touched": tot["blocks_touched"], "blocks_allocated": tot["n_blocks"],
            "scans": len(items), "submaps": len(subs), "tuned": {"pts_per_cta": ppc, "local_blocks": lb},
            "launches_per_step": launches,
            "batched_kernel_ms": kern_ms, "kernel_bytes": kbytes, "sdf_rmse_m": rmse,
            "reset_and_other_ms": ms_b - kern_ms, "pipelined": pipelined,
            "e2e_ms_per_step": e2e_ms, "h2d_bytes_per_step": int(n_points * 12),
            "d2h_bytes_per_step": 48 * len(subs),
            "phases": {"scans": int(len(phases)), "last_tiles_done_ms": float(phases[:, 0].max()),
                       "last_merged_ms": float(phases[:, 1].max()),
                       "median_tiles_done_to_merged_ms": float(np.median(phases[:, 1] - phases[:, 0]))}}


# -------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi, autotune
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    peaks, peak_src = load_peaks()

    if args.workload == "lidar":
        return run_lidar(args, ws, rank, peaks, peak_src)
    wl = make_workload(args.workload, args.frames)
    sm = wl.submaps[0]
    F = len(sm.scans)
    N = sm.scans[0].points.shape[0]
    host = torch.from_numpy(np.stack([s.points for s in sm.scans])).pin_memory()
    pts = host.cuda()
    Ts = [s.T_sub_sensor for s in sm.scans]
    sc0 = sm.scans[0]
    stream = torch.cuda.Stream()
    max_blocks = args.max_blocks

    def prm_of(ppc, lb):
        return cvx.integrate_params(wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range, sc0.sensor,
                                    sc0.height, sc0.width, ppc, lb)

    def make_sub(storage, sets=4, pipelined=True):
        with torch.cuda.stream(stream):
            return cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, storage, max_blocks=max_blocks,
                              stream=stream, pipelined=pipelined, sets=sets)

    def capture(step):
        for _ in range(2):      # warm up the allocator and the kernels outside capture
            step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        torch.cuda.synchronize()
        return g

    def timed(g, steps, warm):
        with torch.cuda.stream(stream):      # replay on the stream the events see
            for _ in range(warm):
                g.replay()
            barrier(ws)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                g.replay()
            e1.record(stream)
            barrier(ws)
        return e0.elapsed_time(e1)

    def profiled(step, steps):
        """Library kernels of `steps` eager steps, each launch bracketed by CUDA
        events on its stream; and the launches one step issues."""
        _capi.cvx_profile_start(1 << 22)
        l0 = _capi.cvx_launch_count()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        n = (_capi.cvx_launch_count() - l0) // steps
        _capi.cvx_profile_stop()
        return _capi.cvx_profile_read(), n

    # ---- the headline path: all frames of the step in one batched persistent
    # launch, four per-scan sets (several frames in flight), shape autotuned
    sample = list(range(min(40, F)))
    if args.ppc == 0:
        tsub = make_sub(cvx.CVX_STORE_F32)
        tuned = autotune.tune_batch([tsub.handle], [(0, pts[f], Ts[f], None, prm_of(0, 0)) for f in sample],
                                    f"{wl.name}|st0|s4|{len(sample)}", reset=lambda: tsub.reset())
        tsub.close()
        args.ppc, args.lb = tuned["pts_per_cta"], tuned["local_blocks"]
        tune_report = tuned["timings"]
    else:
        tune_report = None
    params = prm_of(args.ppc, args.lb)
    scans_all = [(0, pts[f], Ts[f], None, params) for f in range(F)]

    def batched_step(sub, batch, scans):
        sub.reset(stream)
        _capi.cvx_integrate_batch(batch, [sub.handle], scans, stream)

    sub32 = make_sub(cvx.CVX_STORE_F32)
    batch32 = _capi.cvx_batch_create(1, F)
    step32 = lambda: batched_step(sub32, batch32, scans_all)   # noqa: E731
    g32 = capture(step32)
    step32()
    torch.cuda.synchronize()
    c1 = sub32.counters()
    assert _capi.cvx_batch_error(batch32) == 0 and sub32.status() == 0, "device error in the benchmark workload"
    keys, D, W = (t.cpu().numpy() for t in sub32.extract(stream))
    rmse32 = sdf_rmse(wl.scene, keys, D.astype(np.float64), W.astype(np.float64), sm.voxel_size, sm.trunc)

    clocks = Clocks(dev_index)
    clocks.start()
    ms32 = timed(g32, args.steps, args.warmup)
    clk = clocks.stop()
    ms32 = max_over_ranks(ms32, ws)
    prof, launches_per_step = profiled(step32, args.steps)

    # FP16 storage form, same path
    sub16 = make_sub(cvx.CVX_STORE_F16)
    batch16 = _capi.cvx_batch_create(1, F)
    step16 = lambda: batched_step(sub16, batch16, scans_all)   # noqa: E731
    g16 = capture(step16)
    step16()
    torch.cuda.synchronize()
    keys16, D16, W16 = (t.cpu().numpy() for t in sub16.extract(stream))
    D16 = D16.astype(np.float64) * np.float64(np.float32(sm.trunc))
    rmse16 = sdf_rmse(wl.scene, keys16, D16, W16.astype(np.float64), sm.voxel_size, sm.trunc)
    ms16 = max_over_ranks(timed(g16, args.steps, args.warmup), ws)
    prof16, _ = profiled(step16, args.steps)

    # the per-scan path on the same frames (two launches per frame, shape and
    # schedule autotuned), for comparison
    ps_sample = [(pts[f], Ts[f]) for f in range(min(20, F))]
    ps_tuned = {p: autotune.tune_scans(sm.voxel_size, sm.trunc, wl.max_weight, 0, ps_sample, prm_of,
                                       max_blocks=max_blocks, pipelined=p) for p in (False, True)}
    ps_pipe = min(ps_tuned, key=lambda p: ps_tuned[p]["ms"])
    ps_params = prm_of(ps_tuned[ps_pipe]["pts_per_cta"], ps_tuned[ps_pipe]["local_blocks"])
    sub_ps = make_sub(cvx.CVX_STORE_F32, sets=2 if ps_pipe else 1, pipelined=ps_pipe)

    def step_ps():
        sub_ps.reset(stream)
        for f in range(F):
            sub_ps.integrate(pts[f], Ts[f], ps_params, None, stream)
        sub_ps.flush(stream)

    ms_ps = max_over_ranks(timed(capture(step_ps), max(3, args.steps // 2), args.warmup), ws) / max(3, args.steps // 2)
    prof_ps, _ = profiled(step_ps, 2)
    sub_ps.close()

    # end to end through the public API: each step copies its frames from
    # pinned host memory in four chunks on a side stream (double buffered),
    # one batched launch per chunk as its copy lands, counters read back.
    # The copies and launches of a step are captured once as a CUDA graph and
    # replayed (no host work per chunk); the eager sequence is timed beside it
    copy_stream = torch.cuda.Stream()
    n_chunks = 4
    chunk = (F + n_chunks - 1) // n_chunks
    bufs = [torch.empty((chunk, N, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    ev_copied = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    chunk_batches, chunk_scans = [], []
    for c in range(n_chunks):
        f0, f1 = c * chunk, min(F, (c + 1) * chunk)
        chunk_batches.append(_capi.cvx_batch_create(1, chunk))
        chunk_scans.append([(0, bufs[c % 2][f - f0], Ts[f], None, params) for f in range(f0, f1)])

    def e2e_body():
        sub32.reset(stream)
        for b in range(2):
            ev_used[b].record(stream)   # both buffers free once the step's stream gets here
        for c in range(n_chunks):
            b = c % 2
            f0, f1 = c * chunk, min(F, (c + 1) * chunk)
            copy_stream.wait_event(ev_used[b])
            with torch.cuda.stream(copy_stream):
                bufs[b][: f1 - f0].copy_(host[f0:f1], non_blocking=True)
                ev_copied[b].record(copy_stream)
            stream.wait_event(ev_copied[b])
            _capi.cvx_integrate_batch(chunk_batches[c], [sub32.handle], chunk_scans[c], stream)
            ev_used[b].record(stream)

    def e2e_step_eager():
        e2e_body()
        return sub32.counters()   # device -> host read of the step's result

    for _ in range(args.warmup):
        e2e_step_eager()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ce = e2e_step_eager()
    barrier(ws)
    e2e_eager_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, ws)
    assert ce["frames"] == F and ce["valid_points"] == c1["valid_points"]
    torch.cuda.synchronize()
    g_e2e = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_e2e, stream=stream):
        e2e_body()
    torch.cuda.synchronize()

    def e2e_step():
        with torch.cuda.stream(stream):
            g_e2e.replay()
        return sub32.counters()   # device -> host read of the step's result

    for _ in range(args.warmup):
        e2e_step()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ce = e2e_step()
    barrier(ws)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, ws)
    assert ce["frames"] == F and ce["valid_points"] == c1["valid_points"]

    valid = c1["valid_points"]
    obs = c1["observations"]
    merged = c1["voxels_merged"]
    blocks = c1["blocks_touched"]
    new_blocks = c1["n_blocks"]
    tot_valid = sum_over_ranks(valid, ws)
    tot_obs = sum_over_ranks(obs, ws)
    sec32 = ms32 / 1e3 / args.steps
    sec16 = ms16 / 1e3 / args.steps
    pts_s = tot_valid / sec32

    # roofline of the dominant kernel (algorithmic bytes per launch / event time)
    S32 = 8
    bytes_kernel = {
        # the whole frame sequence: points, hash probes and new keys, D/W of the merged voxels
        "batched_kernel": 12 * F * N + 16 * blocks + 12 * new_blocks + 2 * S32 * merged,
        "reset_pools_kernel": S32 * 512 * new_blocks,
    }
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    dom_bytes = bytes_kernel.get(dom, 0.0)
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    path_bytes = 12 * F * N + 2 * S32 * merged + 16 * blocks + S32 * 512 * new_blocks
    path_gbs = path_bytes / sec32 / 1e9

    out = {
        "metric": "TSDF integration points/s (plain FP32, 1 GB300)",
        "value": pts_s,
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms32 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "frames_per_step": F, "points_per_frame": N,
                   "voxel_size_m": sm.voxel_size, "trunc_m": sm.trunc, "weight": "quadratic+linear-dropoff",
                   "storage": "f32",
                   "step": "clear submap + integrate all frames in one batched persistent launch (CUDA graph replay)",
                   "launch_shape": "%d points per tile, %s, 4 per-scan sets" % (
                       args.ppc, "L2 vector reductions" if args.lb < 0 else f"{args.lb or 8} shared block slots"),
                   "autotuned": {"pts_per_cta": args.ppc, "local_blocks": args.lb,
                                 "candidates_ms_%d_frames" % len(sample): tune_report},
                   "l2": "inputs (%.0f MB of points) exceed the 129 MB L2" % (F * N * 12 / 1e6),
                   "parallelism": f"replica x{ws} (one submap sequence per GPU)"},
        "voxel_updates_per_s": tot_obs / sec32,
        "unique_voxel_merges_per_s": sum_over_ranks(merged, ws) / sec32,
        "sdf_rmse_m": rmse32,
        "counts_per_step": {"valid_points": valid, "observations": obs, "voxels_merged": merged,
                            "blocks_touched": blocks, "blocks_allocated": new_blocks},
        "forms": {"fp16_storage": {"points_per_s": tot_valid / sec16, "ms_per_step": ms16 / args.steps,
                                   "speedup_vs_fp32": sec32 / sec16, "sdf_rmse_m": rmse16,
                                   "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof16.items() if v[1]}},
                  "per_scan_path": {"points_per_s": tot_valid / (ms_ps / 1e3), "ms_per_step": ms_ps,
                                    "batched_speedup": ms_ps / (ms32 / args.steps),
                                    "autotuned": {"pts_per_cta": ps_tuned[ps_pipe]["pts_per_cta"],
                                                  "local_blocks": ps_tuned[ps_pipe]["local_blocks"],
                                                  "pipelined": ps_pipe},
                                    "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof_ps.items() if v[1]}}},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": kernel_traffic(dom, args.ppc, args.lb, wl.name), "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms},
        "path_roofline": {"bytes_per_step": path_bytes, "achieved_gbs": path_gbs, "frac": path_gbs / hbm,
                          "block_granular_bytes_per_step": 2 * S32 * 512 * blocks},
        "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items() if v[1]},
        "kernel_share": {k: v[0] / sum(x[0] for x in prof.values()) for k, v in prof.items() if v[1]},
        "e2e": {"value": tot_valid / (e2e_ms / 1e3 / args.steps), "unit": "points/s",
                "h2d_bytes_per_step": int(F * N * 12), "d2h_bytes_per_step": 48,
                "step": "reset + four chunks of frames copied from pinned host memory on a side stream, a batched "
                        "launch per chunk as its copy lands (copies and launches replayed from a CUDA graph), "
                        "counters read back",
                "eager_value": tot_valid / (e2e_eager_ms / 1e3 / args.steps)},
        # graph replays launch the kernels one captured step launched; the
        # library counts every launch it issues (eager step above)
        "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_per_step": launches_per_step,
        "clocks": clk,
    }
    per_scan_sub = lambda storage: make_sub(storage, sets=2 if ps_pipe else 1, pipelined=ps_pipe)   # noqa: E731
    if not args.no_extra:
        out["forms"]["carving"] = carving_form(wl, pts, Ts, stream, args, ws, per_scan_sub, None, timed,
                                               lambda a, b: _capi.cvx_integrate_params.from_buffer_copy(ps_params))
        out["forms"]["esdf"] = esdf_form(sub32, stream, args, peaks)
        out["forms"]["hash_stress"] = hash_stress_form(args)
    if not args.no_learned:
        out["forms"]["learned_weight"] = learned_form(wl, pts, Ts, stream, args, ws, rmse32, ms32 / args.steps,
                                                      make_sub, capture, timed, params)
    if not args.no_lidar:
        out["forms"]["lidar"] = lidar_form(args, ws, rank, peaks, peak_src)
    if not args.no_batched:
        import scenegen as sg
        wl4 = sg.make_c4()
        r4 = bench_multi(wl4, 1, args.steps, args.warmup, ws)
        out["forms"]["batched_fp16"] = {
            "workload": wl4.name + " (1-16 mixed 640x480 / 64x1024 scans each, FP16 storage)",
            "points_per_s": sum_over_ranks(r4["points"], ws) / (r4["ms_per_step"] / 1e3),
            "ms_per_step": r4["ms_per_step"],
            "per_scan_path_points_per_s": sum_over_ranks(r4["points"], ws) / (r4["ms_per_step_per_scan_path"] / 1e3),
            "speedup_vs_per_scan_path": r4["ms_per_step_per_scan_path"] / r4["ms_per_step"],
            "sdf_rmse_m": r4["sdf_rmse_m"], "autotuned": r4["tuned"], "scans": r4["scans"],
            "batched_kernel_ms": r4["batched_kernel_ms"],
            "batched_kernel_gbs": r4["kernel_bytes"] / (r4["batched_kernel_ms"] / 1e3) / 1e9}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
        out["cpu_baseline_parallel"] = cpu_baseline_parallel(wl, args.cpu_seconds / 2)
        err = storage_error_vs_oracle(wl, params, stream, frames=args.error_frames)
        out["forms"]["fp16_storage"]["error_vs_fp64_oracle"] = err["fp16"]
        out["error_fp32_vs_fp64_oracle"] = err["fp32"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    for b in [batch32, batch16] + chunk_batches:
        _capi.cvx_batch_destroy(b)
    for s in (sub32, sub16):
        s.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def carving_form(wl, pts, Ts, stream, args, ws, make_sub, capture, timed, prm_of):
    """Free-space carving on the multiroom frames: every ray traversed from the
    optical centre to trunc behind its point (Sec. III-C), same launch shape,
    FP32, CUDA-graph replay of whole steps like the headline."""
    import torch
    import paper_2410_21149_gb300 as cvx
    prm = prm_of(args.ppc, args.lb)
    prm.flags = cvx._capi.CVX_INTEGRATE_CARVE
    sub = make_sub(cvx.CVX_STORE_F32)
    F = len(Ts)

    def step_c():
        sub.reset(stream)
        for f in range(F):
            sub.integrate(pts[f], Ts[f], prm, None, stream)
        sub.flush(stream)

    for _ in range(2):
        step_c()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step_c()
    torch.cuda.synchronize()
    steps = max(3, args.steps // 5)
    ms = max_over_ranks(timed(g, steps, args.warmup), ws) / steps
    step_c()
    torch.cuda.synchronize()
    c = sub.counters()
    assert sub.status() == 0
    sub.close()
    return {"points_per_s": c["valid_points"] / (ms / 1e3), "voxel_updates_per_s": c["observations"] / (ms / 1e3),
            "ms_per_step": ms, "observations_per_step": c["observations"], "blocks_allocated": c["n_blocks"]}


def esdf_form(sub, stream, args, peaks):
    """Distance field of the integrated multiroom submap (Sec. III-E): time of
    one cvx_compute_esdf call (CUDA events, best of K after W warm-ups), the
    box it sweeps, and its algorithmic bytes: 4 B per box voxel to initialise
    the grid, 8 B per box voxel and axis pass (read + write), 8 B per
    allocated voxel to read D and W, 4 B per allocated voxel written."""
    import torch
    with torch.cuda.stream(stream):
        keys = sub.extract(stream)[0]
        nb = int(keys.shape[0])
        for _ in range(args.warmup):
            sub.esdf(stream=stream)
        ts = []
        for _ in range(max(args.steps, 3)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sub.esdf(stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    k = keys.cpu().numpy()
    box = ((k.max(0) - k.min(0) + 1) * 8).astype(np.int64)
    V, N = int(np.prod(box)), nb * 512
    ms = min(ts)
    nbytes = 4 * V + 3 * 8 * V + 8 * N + 4 * N
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    return {"ms": ms, "blocks": nb, "box_voxels": V, "box": box.tolist(),
            "voxels_out_per_s": N / (ms / 1e3), "box_voxels_per_s": V / (ms / 1e3),
            "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (ms / 1e3) / 1e9,
            "frac_hbm": nbytes / (ms / 1e3) / 1e9 / hbm,
            "site_rule": "W > 0 and |D| <= voxel size; capped at 2 m"}


def hash_stress_form(args, slots_log2=26, load_factors=(0.1, 0.5, 0.85)):
    """The block hash alone (the paper's hash stress test: tens of millions of
    insertions): seeded random block keys (uniform in +-2^19 per axis,
    duplicates allowed) inserted into an empty table of 2^26 slots at each
    load factor, then looked up; best of K timings (CUDA events), table
    cleared between runs."""
    import torch
    from paper_2410_21149_gb300 import _capi
    slots = 1 << slots_log2
    res = {"slots": slots, "key_distribution": "uniform int32 in [-2^19, 2^19) per axis, seeded"}
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    for lf in load_factors:
        n = int(lf * slots)
        coords = torch.randint(-(1 << 19), 1 << 19, (n, 3), dtype=torch.int32, device="cuda", generator=g)
        pool = torch.empty(n, dtype=torch.int32, device="cuda")
        ins, fnd = [], []
        for _ in range(max(3, min(args.steps, 5))):
            h = _capi.cvx_block_hash_create(slots, n)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            _capi.cvx_block_hash_insert(h, coords, pool)
            e1.record()
            _capi.cvx_block_hash_find(h, coords, pool)
            e2.record()
            e2.synchronize()
            st, nb, _ = _capi.cvx_block_hash_info(h)
            assert st == 0, st
            _capi.cvx_block_hash_destroy(h)
            ins.append(e0.elapsed_time(e1))
            fnd.append(e1.elapsed_time(e2))
        res[f"lf{lf}"] = {"keys": n, "distinct": nb, "insert_ms": min(ins), "find_ms": min(fnd),
                          "inserts_per_s": n / (min(ins) / 1e3), "finds_per_s": n / (min(fnd) / 1e3)}
        del coords, pool
    return res


def learned_form(wl, pts, Ts, stream, args, ws, rmse_plain, ms_plain, make_sub, capture, timed, params):
    """Learned per-point weight on the multiroom workload: train the network
    on three other seeded buildings (noisy vs noise-free fused TSDF targets),
    then time per-frame weights + per-point-weight integration of all frames,
    and compare the SDF RMSE with the plain quadratic weight (gate)."""
    import torch
    import scenegen as sg
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi, weights
    sm = wl.submaps[0]
    H, W = sm.scans[0].height, sm.scans[0].width
    t0 = time.perf_counter()
    F, E, M = [], [], []
    for seed in (31, 32, 34):
        noisy = sg.make_c2(seed=seed, n_frames=8, width=W, height=H)
        clean = sg.make_c2(seed=seed, n_frames=8, width=W, height=H, noise=False)
        f, e, m = weights.build_training_set(noisy.submaps[0].scans, clean.submaps[0].scans, sm.voxel_size,
                                             sm.trunc, wl.max_range)
        F.append(f), E.append(e), M.append(m)
    F, E, M = torch.cat(F), torch.cat(E), torch.cat(M)
    E, _ = weights.normalise_targets(E, M)
    model = weights.WeightModel(seed=0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = weights.train(model, F, E, M, steps=1500, batch=65536, lr=3e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    N = sm.scans[0].points.shape[0]
    nf = len(Ts)
    # every frame's per-point weights (features + network fused, all frames in
    # one persistent launch), then all frames in one batched persistent launch
    # with per-point weights: the headline's path and launch shape
    w_all = torch.empty((nf, N), dtype=torch.float32, device="cuda")
    prm = _capi.cvx_integrate_params.from_buffer_copy(params)
    prm.weight_mode = cvx.CVX_W_PER_POINT
    sub = make_sub(cvx.CVX_STORE_F32)
    batch = _capi.cvx_batch_create(1, nf)
    scans_l = [(0, pts[f], Ts[f], w_all[f], prm) for f in range(nf)]

    def step():
        sub.reset(stream)
        _capi.cvx_weight_model_point_weights_frames(model.handle, pts, nf, H, W, 0, wl.max_range, w_all, stream)
        _capi.cvx_integrate_batch(batch, [sub.handle], scans_l, stream)

    g = capture(step)
    step()
    torch.cuda.synchronize()
    assert _capi.cvx_batch_error(batch) == 0 and sub.status() == 0
    keys, D, Wt = (t.cpu().numpy() for t in sub.extract(stream))
    rmse_l = sdf_rmse(wl.scene, keys, D.astype(np.float64), Wt.astype(np.float64), sm.voxel_size, sm.trunc)
    c = sub.counters()
    ms_total = timed(g, args.steps, args.warmup)
    ms = max_over_ranks(ms_total, ws) / args.steps
    _capi.cvx_profile_start(1 << 20)
    step()
    torch.cuda.synchronize()
    _capi.cvx_profile_stop()
    prof = _capi.cvx_profile_read()
    _capi.cvx_batch_destroy(batch)
    sub.close()
    gain = weighting_noise_rmse(model, wl, stream)
    model.close()
    return {"points_per_s": sum_over_ranks(c["valid_points"], ws) / (ms / 1e3),
            "ms_per_step": ms, "speedup_vs_fp32": ms_plain / ms, "sdf_rmse_m": rmse_l, "sdf_rmse_plain_quadratic_m": rmse_plain,
            "gate_keeps_learned": bool(weights.gate(rmse_l, rmse_plain)),
            "noise_rmse_vs_noise_free_fusion": gain,
            "training": {"points": int(F.shape[0]), "steps": 1500, "batch": 65536,
                         "loss_first50": float(np.mean(losses[:50])), "loss_last50": float(np.mean(losses[-50:])),
                         "data_s": t1 - t0, "train_s": t2 - t1},
            "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items() if v[1]}}


def lidar_numbers(args, ws, peaks, peak_src, storage=0, n_scans=2000):
    """LiDAR/MAV workload (64x1024 scans along a 400 m loop, a submap per 50
    scans) through one batched persistent launch per step; the per-scan path
    and the end-to-end copy-in timing beside it."""
    import scenegen as sg
    wl = sg.make_c3(n_scans=n_scans)
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    r = bench_multi(wl, storage, args.steps, args.warmup, ws, max_blocks=1 << 14)
    pts = sum_over_ranks(r["points"], ws)
    ach = r["kernel_bytes"] / (r["batched_kernel_ms"] / 1e3) / 1e9
    return wl, r, {
        "points_per_s": pts / (r["ms_per_step"] / 1e3), "ms_per_step": r["ms_per_step"],
        "voxel_updates_per_s": sum_over_ranks(r["observations"], ws) / (r["ms_per_step"] / 1e3),
        "unique_voxel_merges_per_s": sum_over_ranks(r["voxels_merged"], ws) / (r["ms_per_step"] / 1e3),
        "sdf_rmse_m": r["sdf_rmse_m"],
        "per_scan_path": {"points_per_s": pts / (r["ms_per_step_per_scan_path"] / 1e3),
                          "ms_per_step": r["ms_per_step_per_scan_path"],
                          "batched_speedup": r["ms_per_step_per_scan_path"] / r["ms_per_step"]},
        "roofline": {"bound": "hbm", "kernel": "batched_kernel", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm,
                     "traffic": kernel_traffic("batched_kernel", r["tuned"]["pts_per_cta"], r["tuned"]["local_blocks"],
                                               wl.name) if storage == 0 else None,
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": r["kernel_bytes"], "avg_launch_ms": r["batched_kernel_ms"]},
        "counts_per_step": {k: r[k] for k in ("points", "observations", "voxels_merged", "blocks_touched",
                                              "blocks_allocated", "input_points")},
        "block_granular_bytes_per_step": 2 * (8 if storage == 0 else 4) * 512 * r["blocks_touched"],
        "autotuned": r["tuned"], "batched_phases": r["phases"],
        "e2e": {"value": pts / (r["e2e_ms_per_step"] / 1e3), "unit": "points/s",
                "h2d_bytes_per_step": r["h2d_bytes_per_step"], "d2h_bytes_per_step": r["d2h_bytes_per_step"]},
        "gpu_launches_per_step": r["launches_per_step"],
    }


def lidar_form(args, ws, rank, peaks, peak_src):
    """The LiDAR/MAV workload beside the headline: FP32 (its own roofline,
    e2e, per-scan path) and FP16 storage, with the oracle on a bounded
    prefix."""
    wl, r, res = lidar_numbers(args, ws, peaks, peak_src, storage=0)
    res["workload"] = wl.name + " (40 submaps of 50 scans, batched persistent launch, FP32)"
    _, r16, res16 = lidar_numbers(args, ws, peaks, peak_src, storage=1)
    res["fp16_storage"] = {"points_per_s": res16["points_per_s"], "ms_per_step": res16["ms_per_step"],
                           "speedup_vs_fp32": res["ms_per_step"] / res16["ms_per_step"],
                           "sdf_rmse_m": res16["sdf_rmse_m"], "roofline": res16["roofline"],
                           "autotuned": res16["autotuned"]}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        res["cpu_baseline"] = cpu_baseline(sub_workload(wl, 1), args.cpu_seconds / 2)
        res["cpu_baseline_parallel"] = cpu_baseline_submaps(wl, args.cpu_seconds / 2)
    return res


def sub_workload(wl, n_submaps):
    import copy
    w = copy.copy(wl)
    w.submaps = wl.submaps[:n_submaps]
    return w


def weighting_noise_rmse(model, wl, stream, seeds=(33, 35, 37), frames=40):
    """The gain the weight network is trained for, on held-out buildings: the
    RMS difference between the TSDF fused from noisy scans and the TSDF fused
    from the same scans without noise (same per-ray weights), for constant,
    quadratic and learned weighting with the workload's drop-off; per seed
    and as mean and spread over the seeds."""
    import torch
    import scenegen as sg
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import weights
    sm0 = wl.submaps[0]
    H, W = sm0.scans[0].height, sm0.scans[0].width
    per = {m: [] for m in ("constant", "quadratic", "learned")}
    for seed in seeds:
        noisy = sg.make_c2(seed=seed, n_frames=frames, width=W, height=H).submaps[0]
        clean = sg.make_c2(seed=seed, n_frames=frames, width=W, height=H, noise=False).submaps[0]
        npts = [torch.from_numpy(sc.points).cuda() for sc in noisy.scans]
        cpts = [torch.from_numpy(sc.points).cuda() for sc in clean.scans]
        lw = [weights.learned_point_weights(model, p, H, W, 0, wl.max_range) for p in npts]
        for mode, wm in (("constant", 0), ("quadratic", 1), ("learned", 2)):
            prm = cvx.integrate_params(wm, wl.dropoff, wl.min_range, wl.max_range, 0, H, W)
            out = []
            for pts in (npts, cpts):
                with torch.cuda.stream(stream):
                    sub = cvx.Submap(sm0.voxel_size, sm0.trunc, wl.max_weight, 0, max_blocks=1 << 17, stream=stream)
                for f, sc in enumerate(noisy.scans):
                    # learned: the noisy rays' weights serve both fusions
                    sub.integrate(pts[f], sc.T_sub_sensor, prm, lw[f] if wm == 2 else None, stream)
                out.append(tuple(t.cpu().numpy() for t in sub.extract(stream)))
                sub.close()
            (kn, Dn, Wn), (kc, Dc, Wc) = out
            lut = {tuple(k): b for b, k in enumerate(kc)}
            diffs = []
            for b, k in enumerate(kn):
                bc = lut.get(tuple(k))
                if bc is None:
                    continue
                m = (Wn[b] > 0) & (Wc[bc] > 0) & (np.abs(Dn[b]) < sm0.trunc)
                diffs.append((Dn[b] - Dc[bc])[m].astype(np.float64))
            per[mode].append(float(np.sqrt(np.mean(np.concatenate(diffs) ** 2))))
    return {"seeds": list(seeds), "frames": frames,
            "per_seed_m": per,
            "mean_m": {m: float(np.mean(v)) for m, v in per.items()},
            "spread_m": {m: float(np.std(v)) for m, v in per.items()},
            "learned_vs_quadratic": [l / q for l, q in zip(per["learned"], per["quadratic"])]}


def run_lidar(args, ws, rank, peaks, peak_src):
    """`--workload lidar`: the LiDAR form as the headline line."""
    clocks = Clocks(0)
    clocks.start()
    wl, r, res = lidar_numbers(args, ws, peaks, peak_src, storage=0, n_scans=args.scans)
    clk = clocks.stop()
    out = {
        "metric": "TSDF integration points/s (LiDAR, batched persistent FP32, 1 GB300)",
        "value": res["points_per_s"], "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "submaps": r["submaps"], "scans": r["scans"],
                   "step": "clear all submaps + one batched launch over all scans (CUDA graph replay)",
                   "l2": "inputs (%.0f MB of points) exceed the 129 MB L2" % (r["input_points"] * 12 / 1e6),
                   "launch_shape": r["tuned"], "parallelism": f"replica x{ws}"},
        "gpu_launches": r["launches_per_step"] * args.steps,
        "clocks": clk,
    }
    for k in ("voxel_updates_per_s", "unique_voxel_merges_per_s", "sdf_rmse_m", "per_scan_path", "roofline",
              "counts_per_step", "block_granular_bytes_per_step", "batched_phases", "e2e",
              "gpu_launches_per_step"):
        out[k] = res[k]
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(sub_workload(wl, 1), args.cpu_seconds)
        out["cpu_baseline_parallel"] = cpu_baseline_submaps(wl, args.cpu_seconds / 2)
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- oracle timings
def cpu_baseline(wl, seconds: float):
    """The CPU oracle as it stands (FP64, one thread) on the first frames of
    the same workload: enough frames for about `seconds` of CPU time."""
    import oracle as orc
    sm = wl.submaps[0]
    om = orc.OracleSubmap(sm.voxel_size, sm.trunc, wl.max_weight, bool(wl.storage))
    t0 = time.perf_counter()
    valid = obs = frames = 0
    for sc in sm.scans:
        st = om.integrate(sc.points, sc.T_sub_sensor, None, wl.weight_mode, wl.dropoff, wl.min_range,
                          wl.max_range, sc.sensor)
        valid += st["valid"]
        obs += st["obs"]
        frames += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": valid / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "voxel_updates_per_s": obs / dt,
            "sample": f"first {frames} of {len(sm.scans)} frames of {wl.name} ({valid} valid points, {dt:.1f} s)"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_parallel(wl, seconds: float):
    """The oracle with each frame's sums accumulated by all host cores (OpenMP
    over point chunks, chunk sums added in order) on the first frames of the
    same workload."""
    import oracle as orc
    threads = os.cpu_count() or 1
    sm = wl.submaps[0]
    om = orc.OracleSubmap(sm.voxel_size, sm.trunc, wl.max_weight, bool(wl.storage))
    t0 = time.perf_counter()
    valid = obs = frames = 0
    for sc in sm.scans:
        st = om.integrate_parallel(sc.points, sc.T_sub_sensor, threads, None, wl.weight_mode, wl.dropoff,
                                   wl.min_range, wl.max_range, sc.sensor)
        valid += st["valid"]
        obs += st["obs"]
        frames += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": valid / dt, "unit": "points/s", "cores": threads, "kind": "oracle, OpenMP over point chunks",
            "cpu_model": cpu_model(), "voxel_updates_per_s": obs / dt,
            "sample": f"first {frames} of {len(sm.scans)} frames of {wl.name} ({valid} valid points, {dt:.1f} s)"}


def cpu_baseline_submaps(wl, seconds: float):
    """The oracle on independent submaps at once, one host thread per submap
    (the oracle's calls release the interpreter lock), on the first submaps
    of the workload."""
    import concurrent.futures as cf
    import oracle as orc
    threads = min(os.cpu_count() or 1, len(wl.submaps))
    budget = seconds

    def one(sm):
        om = orc.OracleSubmap(sm.voxel_size, sm.trunc, wl.max_weight, bool(wl.storage))
        t0 = time.perf_counter()
        v = n = 0
        for sc in sm.scans:
            st = om.integrate(sc.points, sc.T_sub_sensor, None, wl.weight_mode, wl.dropoff, wl.min_range,
                              wl.max_range, sc.sensor)
            v += st["valid"]
            n += 1
            if time.perf_counter() - t0 > budget:
                break
        return v, n

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, wl.submaps[:threads]))
    dt = time.perf_counter() - t0
    valid = sum(v for v, _ in res)
    scans = sum(n for _, n in res)
    return {"value": valid / dt, "unit": "points/s", "cores": threads, "kind": "oracle, one thread per submap",
            "cpu_model": cpu_model(),
            "sample": f"first scans of {threads} of {len(wl.submaps)} submaps of {wl.name} ({scans} scans, "
                      f"{valid} valid points, {dt:.1f} s)"}


def storage_error_vs_oracle(wl, params, stream, frames: int = 10):
    """D and W of the GPU path (FP32 storage, and FP16 storage with FP32
    accumulation) after the first `frames` frames of the workload, against the
    FP64 oracle without storage rounding: max and RMS |dD| over voxels with
    W > 0, max relative |dW|."""
    import torch
    import oracle as orc
    import paper_2410_21149_gb300 as cvx
    sm = wl.submaps[0]
    om = orc.OracleSubmap(sm.voxel_size, sm.trunc, wl.max_weight, False)
    for sc in sm.scans[:frames]:
        om.integrate(sc.points, sc.T_sub_sensor, None, wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range,
                     sc.sensor)
    ko, Do, Wo = om.extract()
    res = {}
    for name, storage in (("fp32", 0), ("fp16", 1)):
        with torch.cuda.stream(stream):
            sub = cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, storage, max_blocks=1 << 16, stream=stream)
        for sc in sm.scans[:frames]:
            sub.integrate(torch.from_numpy(sc.points).cuda(), sc.T_sub_sensor, params, None, stream)
        keys, D, W = (t.cpu().numpy() for t in sub.extract(stream))
        sub.close()
        D = D.astype(np.float64) * (np.float64(np.float32(sm.trunc)) if storage else 1.0)
        W = W.astype(np.float64)
        order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
        keys, D, W = keys[order], D[order], W[order]
        if not np.array_equal(keys, ko):
            res[name] = {"error": "block sets differ"}
            continue
        m = Wo > 1e-6
        dD = np.abs(D - Do)[m]
        dW = (np.abs(W - Wo) / np.maximum(Wo, 1e-6))[m]
        res[name] = {"frames": frames, "voxels": int(m.sum()), "max_abs_dD_m": float(dD.max()),
                     "rms_dD_m": float(np.sqrt(np.mean(dD ** 2))), "max_rel_dW": float(dW.max()),
                     "max_abs_dD_over_trunc": float(dD.max() / sm.trunc)}
    return res


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload, args.frames)
    per = max(2.0, args.cpu_seconds / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(wl, per)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(wl, per))
    el = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    print(json.dumps({
        "impl": "reference", "metric": "TSDF integration points/s (plain FP32, 1 GB300)", "value": v,
        "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "step": "bounded sample: first frames of the workload"},
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_steps(args):
    """The benchmark's batched step, eagerly, args.profile_steps times: one
    reset of every submap and one batched launch each, for a profiler to
    capture (a small case: few frames or scans).  Launch shape --ppc/--lb, else
    the shape the autotuner picks on GB300 (multiroom 1024 points per tile,
    LiDAR 2048, both with L2 reductions)."""
    import torch
    import scenegen as sg
    import paper_2410_21149_gb300 as cvx
    from paper_2410_21149_gb300 import _capi
    torch.cuda.set_device(0)
    if args.profile_kernel == "point_weights":
        # the learned form's weight kernel over the frames, untrained network
        from paper_2410_21149_gb300 import weights
        wl = make_workload(args.workload if args.workload != "lidar" else "multiroom", args.frames)
        sm = wl.submaps[0]
        H, W = sm.scans[0].height, sm.scans[0].width
        pts = torch.from_numpy(np.stack([sc.points for sc in sm.scans])).cuda()
        model = weights.WeightModel(seed=0)
        w = torch.empty((len(sm.scans), H * W), dtype=torch.float32, device="cuda")
        for _ in range(args.profile_steps):
            weights.learned_point_weights_frames(model, pts, H, W, sm.scans[0].sensor, wl.max_range, out=w)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(w).all())
        print(json.dumps({"profile_steps": args.profile_steps, "kernel": "point_weights_kernel",
                          "workload": wl.name, "frames": len(sm.scans), "points": int(pts.shape[0] * pts.shape[1])}))
        model.close()
        return
    if args.workload == "lidar":
        wl, max_blocks, ppc = sg.make_c3(n_scans=args.scans), 1 << 14, 2048
    else:
        wl, max_blocks, ppc = make_workload(args.workload, args.frames), 1 << 16, 1024
    if args.profile_shapes:   # "ppc,lb;ppc,lb;...": each shape's launches in turn, in this order
        shapes = [tuple(int(v) for v in x.split(",")) for x in args.profile_shapes.split(";")]
    else:
        shapes = [(args.ppc, args.lb) if args.ppc else (ppc, -1)]
    subs = [cvx.Submap(sm.voxel_size, sm.trunc, wl.max_weight, 0, max_blocks=max_blocks, sets=4)
            for sm in wl.submaps]
    handles = [s.handle for s in subs]
    pts = [(m, torch.from_numpy(np.ascontiguousarray(sc.points)).cuda(), sc)
           for m, sm in enumerate(wl.submaps) for sc in sm.scans]
    batch = _capi.cvx_batch_create(len(subs), len(pts))
    for ppc, lb in shapes:
        scans = [(m, p, sc.T_sub_sensor, None,
                  cvx.integrate_params(wl.weight_mode, wl.dropoff, wl.min_range, wl.max_range, sc.sensor,
                                       sc.height, sc.width, ppc, lb)) for m, p, sc in pts]
        for _ in range(args.profile_steps):
            _capi.cvx_reset_submaps(handles)
            _capi.cvx_integrate_batch(batch, handles, scans)
        torch.cuda.synchronize()
        assert _capi.cvx_batch_error(batch) == 0 and all(s.status() == 0 for s in subs)
        c = [s.counters() for s in subs]
        print(json.dumps({"profile_steps": args.profile_steps, "workload": wl.name, "submaps": len(subs),
                          "scans": len(scans), "launch_shape": [ppc, lb],
                          "input_points": sum(int(x[1].shape[0]) for x in scans),
                          "counts": {k: sum(x[k] for x in c) for k in c[0]}}))
    _capi.cvx_batch_destroy(batch)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="multiroom", choices=["multiroom", "room", "lidar"])
    ap.add_argument("--scans", type=int, default=2000, help="LiDAR scans (lidar workload)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched form (multiroom)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-weight form (multiroom)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the carving, ESDF and hash-stress forms (multiroom)")
    ap.add_argument("--no-lidar", action="store_true", help="skip the LiDAR form (multiroom)")
    ap.add_argument("--error-frames", type=int, default=10,
                    help="frames of the storage-error comparison against the oracle (CPU leg)")
    ap.add_argument("--frames", type=int, default=200)
    ap.add_argument("--ppc", type=int, default=0, help="points per CTA tile (0: autotuned)")
    ap.add_argument("--lb", type=int, default=0, help="shared block slots per CTA (-1: global atomics)")
    ap.add_argument("--pipelined", type=int, default=-1, choices=[-1, 0, 1],
                    help="pipelined submaps on the per-scan path (-1: autotuned with the launch shape)")
    ap.add_argument("--max-blocks", type=int, default=1 << 18)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiler mode: run only the batched step of --workload this many times, eagerly "
                         "(--frames frames, or --scans LiDAR scans), no timing and no other forms")
    ap.add_argument("--profile-shapes", default="",
                    help="profiler mode: launch shapes 'ppc,lb;ppc,lb;...' run in turn, --profile-steps each")
    ap.add_argument("--profile-kernel", default="batched", choices=["batched", "point_weights"],
                    help="profiler mode: the batched step, or the learned form's weight kernel over --frames frames")
    args = ap.parse_args()
    if args.profile_steps > 0:
        return profile_steps(args)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
