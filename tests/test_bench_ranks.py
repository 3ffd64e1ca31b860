"""The benchmark's host logic on CPU: the multi-rank aggregation (gloo, two
processes: the step time is the maximum over ranks and the value counts every
rank's products), the reference arm on rank 0 only, and the spawned processes of
the CPU oracle baseline (timed together; a failed worker is reported, not waited
for).  No GPU is used."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, _ = bench.dist_env()
ms, value = bench.job_value(10.0 * (rank + 1), 1024, world, dist, "cpu")
print(json.dumps({"rank": rank, "ms": ms, "value": value}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_value_takes_the_slowest_rank_over_gloo():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 20.0
        assert abs(o["value"] - 2 * 1024 / 0.020) < 1e-6


def test_job_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_value(12.5, 1024, 1)
    assert ms == 12.5 and abs(value - 1024 / 0.0125) < 1e-9


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_cpu_baseline_processes_time_together():
    """The CPU baseline's spawned processes (one BLAS thread each) all finish a sample; the
    rate adds their products per second."""
    sys.path.insert(0, ROOT)
    import bench
    done, el, rate = bench.cpu_oracle_rate(0.3, 2, workload="l96_small")
    assert done >= 2 and el >= 0.3
    assert rate > 0 and rate >= done / el * 0.5


def test_cpu_baseline_reports_a_failed_worker_instead_of_waiting():
    sys.path.insert(0, ROOT)
    import time
    import bench
    t0 = time.time()
    with pytest.raises(RuntimeError):
        bench.cpu_oracle_rate(0.1, 2, workload="no_such_workload")
    assert time.time() - t0 < 60
