"""One rank of the world_size > 1 checks, launched by
tests/test_multirank_cpu.py through torch.distributed.run on the gloo backend
(CPU only).

View sharding of one batch: every rank renders its block of the views
(paper_2512_08498_gb300.sharding.shard_views) with the CPU oracle against
the same Gaussians, and the ranks' parameter gradients are summed by the one
all-reduce of a flat buffer (allreduce_grads).  Rank 0 then renders the whole
batch in one oracle call and records how far the summed gradients and the
ranks' own pose gradients are from it.  The bench's timing reductions
(max over ranks, whole-job rate) are exercised too.  Rank 0 writes what it
saw to the JSON path given as the only argument."""
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
import oracle
from paper_2512_08498_gb300 import scenes
from paper_2512_08498_gb300.scenes import look_from, pinhole
from paper_2512_08498_gb300.sharding import GradBuffer, allreduce_grads, shard_views

NAMES = ["means", "log_scales", "quats", "opacity_logits", "sh"]


def batch():
    n = 300
    rng = np.random.default_rng(4)
    views = [pinhole(40, 30, f=40.0),
             pinhole(36, 28, f=36.0, viewmat=look_from([0.1, -0.05, -0.2], yaw_deg=6.0)),
             pinhole(48, 20, f=44.0, viewmat=look_from([-0.1, 0.05, 0.1], yaw_deg=-8.0),
                     subset=np.sort(rng.choice(n, n // 2, replace=False)).astype(np.uint32)),
             pinhole(24, 24, f=30.0, viewmat=look_from([0.0, 0.1, -0.1], roll_deg=15.0))]
    return scenes.random_scene(4, n, views, 2, bg=(0.1, 0.2, 0.3))


def sub_scene(sc, a, b):
    return scenes.Scene(sc.name, sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh, sc.sh_degree,
                        sc.views[a:b], tile=sc.tile, bg=sc.bg, target_seed=sc.target_seed)


def upstream(sc, o, targets, first):
    """Per view of o's scene (view `first` of the batch onward): the L1
    gradient against the batch's targets and seeded depth/alpha terms."""
    ref = o.forward()
    d_rgb, d_dep, d_alp = [], [], []
    for i, v in enumerate(o.views):
        g = np.random.default_rng(100 + first + i)
        n = 3 * v.width * v.height
        d_rgb.append(np.sign(ref["rgb"][i] - targets[first + i]) / n)
        d_dep.append(0.05 * g.standard_normal((v.height, v.width)) / n)
        d_alp.append(0.3 * g.standard_normal((v.height, v.width)) / n)
    return d_rgb, d_dep, d_alp


def main(out_path):
    ws, rank, _ = bench._dist()
    dist.init_process_group("gloo")
    sc = batch()
    targets = sc.targets()
    a, b = shard_views(sc.views, rank, ws)
    buf = GradBuffer(sc.n, sc.sh_degree, "cpu", dtype=torch.float64)
    pose = np.zeros((b - a, 6))
    if b > a:
        o = oracle.Oracle(sub_scene(sc, a, b))
        g = o.backward(*upstream(sc, o, targets, a))
        for name, t in zip(NAMES, buf.tensors()):
            t.copy_(torch.from_numpy(np.asarray(g[name]).reshape(t.shape)))
        pose = g["pose"]
    allreduce_grads(buf)
    poses = [None] * ws
    dist.all_gather_object(poses, (a, b, pose.tolist()))
    local_ms = 10.0 + 5.0 * rank            # rank r "took" 10 + 5 r ms
    ms = bench.max_over_ranks(local_ms, ws, "cpu")
    rate = len(sc.views) / (ms / 1000.0)   # the whole batch over the slowest rank
    dist.barrier()
    if rank == 0:
        full = oracle.Oracle(sc)
        gf = full.backward(*upstream(sc, full, targets, 0))
        errs = {}
        for name, t in zip(NAMES, buf.tensors()):
            ref = np.asarray(gf[name]).reshape(-1)
            errs[name] = float(np.linalg.norm(t.numpy().reshape(-1) - ref) / np.linalg.norm(ref))
        pose_err = 0.0
        for (pa, pb, pp) in poses:
            if pb > pa:
                d = np.asarray(pp) - gf["pose"][pa:pb]
                pose_err = max(pose_err, float(np.abs(d).max() / np.abs(gf["pose"]).max()))
        with open(out_path, "w") as f:
            json.dump({"ws": ws, "shards": [(p[0], p[1]) for p in poses], "grad_rel_l2": errs,
                       "pose_rel": pose_err, "ms": ms, "rate": rate, "views": len(sc.views)}, f)
    dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
