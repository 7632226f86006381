"""One rank of the two-rank replica check (run by test_multiprocess.py):
bench.py's own rendezvous, barrier and max-over-ranks reduction over gloo;
prints this rank's view as one JSON line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    ws, rank, local = bench.dist_init()
    bench.barrier(ws)
    # each replica times its own steps; the job's time is the slowest rank's
    ms = 100.0 * (rank + 1)
    ms_max = bench.max_over_ranks(ws, ms)
    steps = 3
    value = ws * steps / (ms_max / 1e3)
    bench.barrier(ws)
    print(json.dumps({"rank": rank, "world_size": ws, "local": local, "ms_max": ms_max, "value": value}))
    import torch.distributed as dist
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
