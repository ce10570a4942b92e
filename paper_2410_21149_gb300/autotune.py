"""Autotuner for the integration kernels' launch shape.

Searches, for one kind of scan (sensor model, image size, voxel size,
truncation, weighting, storage), the points per CTA tile (256 threads, so
points per warp = tile / 8) and the number of shared-memory block slots per
CTA (``local_blocks``; -1 = global vector atomics only), timing each candidate
on sample scans with CUDA events around the library's kernel launches.  The
winner is cached in a JSON file keyed by the device name and the scan
signature (``$COVOX_TUNE_CACHE`` or ``~/.cache/covox_gb300/autotune.json``).

The timed work runs through the same C entry points as production calls
(per-scan or batched); the tuner only chooses parameters.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

from . import _capi

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (256, 2), (256, 4), (256, 8), (256, -1), (512, 4), (512, 8), (512, -1), (1024, 4), (1024, 8), (1024, -1))
# the batched persistent launch takes whole tiles as work items: larger tiles amortise an item's
# dependency check and queue atomic
BATCH_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (256, -1), (256, 2), (512, -1), (512, 4), (1024, -1), (1024, 4), (2048, -1), (2048, 8))

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("COVOX_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "covox_gb300", "autotune.json")


def _load() -> Dict[str, dict]:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: Dict[str, dict]) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def signature(mode: str, sensor: int, height: int, width: int, voxel_size: float, trunc: float,
              weight_mode: int, dropoff: int, storage: int) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    return (f"{dev}|{mode}|s{sensor}|{height}x{width}|vs{voxel_size:.4f}|tr{trunc:.4f}|"
            f"w{weight_mode}|d{dropoff}|st{storage}")


def _time_ms(run, repeats: int) -> float:
    """Best of `repeats` timings of run(), recorded once as a CUDA graph and
    replayed (host launch overhead would otherwise blur candidates whose GPU
    times are close); eager if the run cannot be captured."""
    import torch
    run()                                   # warm-up (allocations, first touch)
    torch.cuda.synchronize()
    replay = run
    graph = None
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            run()
        replay = graph.replay
    except RuntimeError:
        graph = None
        torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        replay()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del graph
    return best


def tune(key: str, make_run, candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
         repeats: int = 3, force: bool = False) -> Dict[str, float]:
    """Time make_run(pts_per_cta, local_blocks)() for every candidate; return
    and cache {"pts_per_cta", "local_blocks", "ms", "timings"}."""
    with _lock:
        cache = _load()
        if not force and key in cache:
            return cache[key]
    timings = {}
    for ppc, lb in candidates:
        timings[f"{ppc},{lb}"] = _time_ms(make_run(ppc, lb), repeats)
    best = min(timings, key=timings.get)
    ppc, lb = (int(x) for x in best.split(","))
    res = {"pts_per_cta": ppc, "local_blocks": lb, "ms": timings[best], "timings": timings}
    with _lock:
        cache = _load()
        cache[key] = res
        _store(cache)
    return res


def tune_scans(voxel_size: float, trunc: float, max_weight: float, storage: int, scans: Sequence[tuple],
               params_fn, max_blocks: int = 1 << 16, force: bool = False,
               candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
               pipelined: bool = False) -> Dict[str, float]:
    """Per-scan path on a scratch submap.  scans: [(points tensor, T)];
    params_fn(ppc, lb) -> cvx_integrate_params.  pipelined: time a pipelined
    submap (each scan's merge overlapped with the next scan; flushed at the
    end), cached under its own key."""
    from . import Submap
    p0 = params_fn(0, 0)
    key = signature("scan", p0.sensor, p0.height, p0.width, voxel_size, trunc, p0.weight_mode,
                    p0.dropoff, storage) + ("|p1" if pipelined else "")
    sub = Submap(voxel_size, trunc, max_weight, storage, max_blocks=max_blocks, pipelined=pipelined)

    def make_run(ppc, lb):
        prm = params_fn(ppc, lb)

        def run():
            sub.reset()
            for pts, T in scans:
                sub.integrate(pts, T, prm)
            sub.flush()
        return run

    try:
        return tune(key, make_run, candidates, force=force)
    finally:
        sub.close()


def tune_batch(maps: List[int], scans: List[tuple], key_parts: str, force: bool = False,
               candidates: Iterable[Tuple[int, int]] = BATCH_CANDIDATES, reset=None) -> Dict[str, float]:
    """Batched path.  maps: submap handles; scans: [(map index, points, T, pw,
    params)] whose params' pts_per_cta / local_blocks are replaced by each
    candidate; reset() clears the submaps between runs."""
    import torch
    key = f"{torch.cuda.get_device_name()}|batch|{key_parts}"
    batch = _capi.cvx_batch_create(len(maps), len(scans))

    def make_run(ppc, lb):
        cand = []
        for (m, pts, T, pw, prm) in scans:
            q = _capi.cvx_integrate_params.from_buffer_copy(prm)
            q.pts_per_cta, q.local_blocks = ppc, lb
            cand.append((m, pts, T, pw, q))

        def run():
            if reset is not None:
                reset()
            _capi.cvx_integrate_batch(batch, maps, cand)
        return run

    try:
        return tune(key, make_run, candidates, force=force)
    finally:
        torch.cuda.synchronize()
        _capi.cvx_batch_destroy(batch)
