"""Free-space carving (rays cast from the optical centre, Sec. III-C) against
the oracle: block sets bit-exact, D within 1e-5 m, W within 1e-4 relative,
exact observation counts; per-scan, pipelined and batched paths."""
import numpy as np
import pytest

import scenegen as sg
from _harness import compare, run_gpu, run_gpu_batched, run_oracle

pytestmark = pytest.mark.gpu

D_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("lb,pipelined", [(0, False), (-1, False), (4, True)])
def test_room_carving(lb, pipelined):
    wl = sg.make_c1(n_frames=4)
    g = run_gpu(wl, pipelined=pipelined, local_blocks=lb, carve=True)[0]
    o = run_oracle(wl, carve=True)[0]
    r = compare(g, o, D_TOL)
    assert g[3]["observations"] == o[3]["obs"] and g[3]["valid_points"] == o[3]["valid"]
    plain = run_oracle(wl)[0]
    assert r["blocks"] > len(plain[0])             # carving reaches blocks the band does not


def test_multiroom_carving_dropoff():
    wl = sg.make_c2(n_frames=2, width=320, height=240, dropoff=1)
    compare(run_gpu(wl, carve=True)[0], run_oracle(wl, carve=True)[0], D_TOL)


def test_lidar_scan_carving():
    wl = sg.make_c3(n_scans=1, scans_per_submap=1, n_boxes=300)
    g = run_gpu(wl, local_blocks=-1, carve=True)[0]
    o = run_oracle(wl, carve=True)[0]
    compare(g, o, D_TOL)
    assert g[3]["observations"] == o[3]["obs"]


def test_batched_carving():
    wl = sg.make_c1(n_frames=4)
    g = run_gpu_batched(wl, carve=True)
    o = run_oracle(wl, carve=True)
    for a, b in zip(g, o):
        compare(a, b, D_TOL)
