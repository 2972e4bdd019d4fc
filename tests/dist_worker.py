"""One rank of the two-rank gloo test of bench.py's multi-rank host logic
(run as a subprocess by tests/test_bench_dist.py, with the torchrun
environment variables set).  Prints one JSON line with what this rank saw."""
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    rank, local, world, dist = bench.dist_setup(2, backend="gloo")
    # rank r took (3 + r) ms for 100 (r + 1) particle steps and 7 events
    agg = bench.aggregate(dist, 3.0 + rank, 100.0 * (rank + 1), 7.0)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        printed = bench.emit({"value": agg["value"], "rank": rank}, rank)
        if rank != 0:
            # the reference arm's other ranks return before any work
            bench.run_reference(None, rank, world, None)
    seed = bench.replica_seed(100, rank)
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps({"rank": rank, "local": local, "world": world, "agg": agg,
                      "printed": printed, "out": buf.getvalue(), "seed": seed}))


if __name__ == "__main__":
    main()
