"""World-size-2 checks of the multi-rank path on CPU (gloo).

One batch is sharded by views over the ranks; every rank holds the Gaussians
and renders its views; the only exchange is one all-reduce (sum) of the
parameter gradients.  These tests launch two ranks with torch.distributed.run
exactly as a multi-GPU bench run is launched, on the gloo backend, with the
CPU oracle standing in for each rank's renderer: the summed shard gradients
must equal the single-process oracle over all views, the ranks' pose
gradients the corresponding rows, and the bench's timing reductions and the
rank-0-only output of the oracle arm must hold."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, nproc=2, timeout=240):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_view_shards_sum_to_the_whole_batch(tmp_path, oracle_lib):
    out = tmp_path / "r0.json"
    p = _torchrun([os.path.join("tests", "_multirank_worker.py"), str(out)])
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    r = json.loads(out.read_text())
    assert r["ws"] == 2
    # contiguous blocks covering every view once
    assert r["shards"][0][0] == 0 and r["shards"][0][1] == r["shards"][1][0] and r["shards"][1][1] == r["views"]
    assert all(b > a for a, b in r["shards"])
    # FP64 sums in another order: equal to rounding
    for name, e in r["grad_rel_l2"].items():
        assert e <= 1e-12, (name, e)
    assert r["pose_rel"] <= 1e-12
    # the slowest rank sets the step time; the rate counts all views of the batch
    assert r["ms"] == pytest.approx(15.0)
    assert r["rate"] == pytest.approx(r["views"] / 0.015)


def test_shard_bounds():
    sys.path.insert(0, ROOT)
    from paper_2512_08498_gb300.sharding import shard_bounds
    import bench
    assert shard_bounds([1] * 6, 1) == [0, 6]
    assert shard_bounds([1] * 6, 2) == [0, 3, 6]
    assert shard_bounds([1] * 6, 3) == [0, 2, 4, 6]
    # pixel-balanced: one large view against three small ones
    assert shard_bounds([300, 100, 100, 100], 2) == [0, 1, 4]
    # more ranks than views: some ranks render nothing, every view once
    b = shard_bounds([1] * 6, 8)
    assert b[0] == 0 and b[-1] == 6 and all(y >= x for x, y in zip(b, b[1:]))
    assert sum(y - x for x, y in zip(b, b[1:])) == 6
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7, 1) == 7.0


def test_reference_arm_prints_on_rank0_only(oracle_lib):
    p = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--workload", "small_box",
                   "--scale", "0.05", "--steps", "1", "--warmup", "0"])
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
