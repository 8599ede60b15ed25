"""One rank of the whole-job timing test (run by test_bench_dist.py as a
separate process; gloo on the CPU): each rank reports a different local time
and gets back the slowest rank's time and the whole job's rate."""
import json
import os
import sys

import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    ms, rate = bench.whole_job_rate(local_ms, 1.0e6, world, "cpu")
    with open(sys.argv[1], "w") as f:
        json.dump({"ms": ms, "rate": rate}, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
