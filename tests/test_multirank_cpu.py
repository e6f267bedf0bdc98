"""World-size-2 checks of the multi-rank host logic on CPU (gloo).

The rasterizer shards across GPUs by giving each rank its own independent
batch (weak scaling): nothing on the data path is exchanged, only the step
time (max over ranks) and the reported counts (sums).  These tests launch two
ranks with torch.distributed.run exactly as a multi-GPU bench run is
launched, on the gloo backend, and check the shard seeds, the reductions and
the rank-0-only output of the oracle arm."""
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


def test_shards_reductions_and_rate(tmp_path):
    out = tmp_path / "r0.json"
    p = _torchrun([os.path.join("tests", "_multirank_worker.py"), str(out)])
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    r = json.loads(out.read_text())
    assert r["ws"] == 2
    # each rank renders its own batch: the shards differ
    assert len(set(r["digests"])) == 2
    # the slowest rank sets the step time; counts add up
    assert r["ms"] == pytest.approx(15.0)
    assert r["pairs"] == pytest.approx(3000.0)
    # whole-job rate: both ranks' views over the slowest rank's time
    assert r["rate"] == pytest.approx(2 * r["views"] / 0.015)


def test_shard_seed_offsets_are_distinct():
    sys.path.insert(0, ROOT)
    import bench
    offs = [bench.shard_seed_offset(r) for r in range(8)]
    assert len(set(offs)) == 8 and offs[0] == 0
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7, 1) == 7.0
    assert bench.job_rate(6, 4, 0.5) == pytest.approx(48.0)


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
