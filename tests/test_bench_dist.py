"""The bench's multi-rank path on CPU: two gloo ranks check that the whole-job
figure is the bytes all ranks processed over the slowest rank's time, and that
the reference arm does its work on rank 0 only."""
import io
import json
import os
import socket
import subprocess
import sys
import contextlib

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
import bench
rank = dist.get_rank()
ms_local = [2.0, 3.0][rank]
bytes_local = [1.0e9, 2.0e9][rank]
gbps, ms = bench.whole_job_gbps(bytes_local, ms_local, dist.get_world_size(), device="cpu")
mx = bench.reduce_max([5.0, 4.0][rank], dist.get_world_size(), device="cpu")
print(json.dumps({"rank": rank, "gbps": gbps, "ms": ms, "max": mx}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_whole_job_aggregation_two_gloo_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank), REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        # (1e9 + 2e9) bytes over the slower rank's 3 ms
        assert o["ms"] == 3.0
        assert o["gbps"] == pytest.approx(3.0e9 / 3.0e-3 / 1e9)
        assert o["max"] == 5.0


def test_single_rank_aggregation_is_local():
    import bench
    gbps, ms = bench.whole_job_gbps(4.0e9, 2.0, 1)
    assert ms == 2.0 and gbps == pytest.approx(2000.0)


def test_reference_arm_only_on_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1",
                                                   "--warmup", "3"]))
    assert rc == 0 and buf.getvalue() == ""
