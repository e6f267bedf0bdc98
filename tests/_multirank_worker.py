"""One rank of the world_size > 1 host-logic check, launched by
tests/test_multirank_cpu.py through torch.distributed.run on the gloo backend
(CPU only).  It exercises the pieces of bench.py that differ between one and
several ranks: the per-rank shard seed, the max-over-ranks step time, the
sum-over-ranks pair count and the whole-job rate.  Rank 0 writes what it saw
to the JSON path given as the only argument."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np
import torch
import torch.distributed as dist

import bench


def main(out_path):
    ws, rank, _ = bench._dist()
    dist.init_process_group("gloo")
    scene = bench.build_workload("small_box", 0.05, bench.shard_seed_offset(rank))
    digest = hashlib.sha256(np.ascontiguousarray(scene.means).tobytes()).hexdigest()
    # test-only exchange of what each shard holds (bench itself exchanges only timings)
    digests = [None] * ws
    dist.all_gather_object(digests, digest)
    local_ms = 10.0 + 5.0 * rank            # rank r "took" 10 + 5 r ms
    ms = bench.max_over_ranks(local_ms, ws, "cpu")
    pairs = bench.sum_over_ranks(1000 * (rank + 1), ws, "cpu")
    rate = bench.job_rate(len(scene.views), ws, ms / 1000.0)
    dist.barrier()
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"ws": ws, "digests": digests, "ms": ms, "pairs": pairs, "rate": rate,
                       "views": len(scene.views), "n": scene.n}, f)
    dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
