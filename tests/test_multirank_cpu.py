"""The multi-process path of bench.py on CPU (gloo, world size 2): the
whole-job value is the units of all ranks over the slowest rank's time,
with no data-path collective; rank 0 alone prints."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys, json, time
    sys.path.insert(0, {root!r})
    import bench
    ws, rank, local = bench.dist_setup("gloo")
    units = 1000.0 * (rank + 1)          # uneven work per rank
    ms = 10.0 + 5.0 * rank               # rank 1 is slower
    bench.barrier(ws)
    tot = bench.sum_over_ranks(units, ws)
    slow = bench.max_over_ranks(ms, ws)
    if rank == 0:
        print(json.dumps({{"value": tot / (slow / 1e3), "tot": tot, "slow": slow, "ws": ws}}))
    import torch.distributed as dist
    dist.destroy_process_group()
""")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_gloo_reductions(tmp_path):
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT))
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    import json
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["ws"] == 2 and line["tot"] == 3000.0 and line["slow"] == 15.0
    assert abs(line["value"] - 3000.0 / 0.015) < 1e-6
    assert outs[1][0].strip() == ""          # only rank 0 prints


def test_reference_arm_nonzero_ranks_exit_quietly():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
