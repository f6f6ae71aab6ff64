"""One rank of the two-rank CPU check of bench.py's multi-rank logic; run
under torch.distributed.run (gloo, 127.0.0.1).  Prints one JSON line."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, world, _ = bench.dist_env()
    dist.init_process_group("gloo")
    step_ms = 10.0 + 5.0 * rank  # each rank's own step time; the slowest one counts
    slowest = bench.max_over_ranks(step_ms, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(7, rank))
    line = json.dumps({"rank": rank, "world": world, "max_ms": slowest, "seeds": seeds,
                       "value": bench.job_keys_per_s(world, 1000, slowest)}) + "\n"
    for r in range(world):  # one rank at a time, one write per line: lines do not interleave
        if r == rank:
            os.write(1, line.encode())
        dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
