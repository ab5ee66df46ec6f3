"""One rank of the benchmark's N-replica timing protocol on the CPU (gloo), launched by
torch.distributed.run from the multi-process tests.  Each rank takes a different time, solves a
different keyframe, and writes what it saw to <outdir>/rank<r>.json; the report goes to
<outdir>/report<r>.txt, which only rank 0 fills."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bench  # noqa: E402


def main(outdir: str, units: float):
    ranks = bench.Ranks("gloo")
    ranks.barrier()
    own_ms = 10.0 + 30.0 * ranks.rank
    slowest = ranks.max_ms(own_ms)
    value = ranks.throughput(units, slowest)
    prob = bench.make_problem(ranks.rank)
    ranks.barrier()
    seen = dict(rank=ranks.rank, world=ranks.world, local=ranks.local, own_ms=own_ms, max_ms=slowest, value=value,
                residuals=bench.residuals_per_step(prob), keyframe_sum=float(np.asarray(prob.keyframe, np.float64).sum()))
    with open(os.path.join(outdir, f"rank{ranks.rank}.json"), "w") as f:
        json.dump(seen, f)
    with open(os.path.join(outdir, f"report{ranks.rank}.txt"), "w") as f:
        ranks.report({"value": value, "n_gpus": ranks.world}, out=f)
    ranks.close()


if __name__ == "__main__":
    main(sys.argv[1], float(sys.argv[2]))
