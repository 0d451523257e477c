"""Replica timing across ranks (CPU, gloo, world size 2): bench.py runs one independent RVE per
rank and reports the units all ranks processed over the slowest rank's time."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_time_and_all_units(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}",
           os.path.join(ROOT, "tests", "multirank_worker.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1", RF_MULTIRANK_OUT=str(tmp_path))
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{i}.json").read_text()) for i in range(2)]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["world"] == 2 and l["local"] == l["rank"]
        assert l["ms"] == 150.0 and l["units"] == 30.0


def test_one_process_passes_its_own_numbers_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 12.5, 7, "cpu") == (12.5, 7.0)
