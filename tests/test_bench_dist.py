"""bench.py's multi-rank aggregation (gloo, world size 2, CPU): the job's
time is the slowest rank's, and its rate counts the units of every rank."""
import json
import os
import socket
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_whole_job_rate_two_ranks(tmp_path):
    port = free_port()
    procs, outs = [], []
    for rank in range(2):
        out = str(tmp_path / f"rank{rank}.json")
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "dist_bench_worker.py"),
                                       out], env=env))
        outs.append(out)
    for p in procs:
        assert p.wait(timeout=120) == 0
    for out in outs:
        r = json.load(open(out))
        assert r["ms"] == 150.0  # the slower rank
        assert r["rate"] == 2 * 1.0e6 / 0.150


def test_whole_job_rate_one_rank():
    import bench
    assert bench.whole_job_rate(200.0, 5.0e5, 1, "cpu") == (200.0, 5.0e5 / 0.2)
