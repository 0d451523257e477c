"""One rank of the two-rank CPU check of bench.py's replica timing (launched by torchrun from
test_multirank.py with the gloo backend; not a test module itself)."""

import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    ws, rank, local = bench.dist_info()
    dist.init_process_group("gloo")
    # rank r timed 100 + 50 r ms for 10 (r + 1) units of work
    ms, units = bench.combine_ranks(dist, 100.0 + 50.0 * rank, 10 * (rank + 1), "cpu")
    # one file per rank: the ranks share stdout, where their lines can interleave
    out = os.path.join(os.environ["RF_MULTIRANK_OUT"], f"rank{rank}.json")
    with open(out, "w") as fh:
        json.dump({"rank": rank, "world": ws, "local": local, "ms": ms, "units": units}, fh)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
