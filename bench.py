"""Benchmark: batched fwd+bwd rasterization of a multi-camera rig on GB300.

One step = forward render of every view of the batch, the L1 photometric
loss gradient against the seeded target images, and the backward pass to all
Gaussian parameters and the per-view se(3) poses: one pass of the whole
rasterization hot path (projection, tile lists, sort, ranges, compositing and
their adjoints) of one iteration of the paper's per-keyframe optimisation
(Sec. 3.3, Table 3).  The optimizer's parameter update, which consumes these
gradients, is not part of that path.

Default workload: the 6-camera rig batch (1M Gaussians in a 60 m street
corridor, SH degree 3, six 1600x900 cameras yawed 60 degrees apart) rendered
in one batched call.  Metric: views/s (fwd+bwd); also Gaussian-pixel pairs/s,
the same batch as six sequential single-view calls, and the dominant kernel's
fraction of its roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): the batch is sharded by views -- every rank holds the
Gaussians and renders a contiguous block of the views -- and each step ends
with one all-reduce (sum) of the parameter gradients (strong scaling of the
batch); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "fwd+bwd rasterized views/s (batched rig)"
UNIT = "views/s"

# Algorithmic work of the blend kernels: the (pixel, entry) pairs that are
# actually composited (alpha >= 1/255, before the stop) -- the pairs any
# implementation has to evaluate -- times the FP32 operations one such pair
# needs, counted from the blend arithmetic.  Forward: offset (2) + quadratic
# form (5) + P>0 test (1) + exp2 (clamp 1, two roundings, reduce 1, degree-7 Horner
# 7, scale 2) + alpha (2) + two threshold tests (2) + transmittance (2) +
# weight and colour/depth accumulation (5) + transmittance update (1) = 33.  Backward: the forward's
# recompute up to the alpha test (24) + 1 - alpha and its reciprocal (2) +
# transmittance recovery and weight (2) + dL/dalpha with the suffix sums
# folded into one scalar (dC.c + dD z: 4, T_k x - X / (1 - alpha): 2) +
# colour/depth gradients (4) + opacity/conic/mean partials (7; the record's
# coefficients are applied once per record) + suffix update (1) + the warp
# reduction's share (1) = 47.  Pairs that are examined but not
# composited are overhead, not counted.
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# blend kernels, from one ncu capture of the default workload and launch
# configuration.  Reported as the roofline's "traffic" only for that workload
# and configuration; to be re-captured whenever those kernels change.
PROFILED_DRAM_BYTES = {"blend_bwd": 403.9e6, "blend_fwd": 405.6e6}
PROFILED_CONFIG = ("rig6", 1.0, (16, 16), 256, 128)   # workload, scale, tile, batch, backward batch

OPS_FWD_PAIR = 33
OPS_BWD_PAIR = 47
# Operations the kernels execute per composited pair.  The forward evaluates
# the contract's 2^x (the decisions depend on it): 33.  The backward takes
# alpha's value from one ex2.approx instead of the 13-operation polynomial
# and re-takes the two decisions with the polynomial only near a threshold,
# which costs one proximity test (subtract, multiply-add, compare: 3):
# 47 - 13 + 1 + 3 = 38.
OPS_FWD_PAIR_EXEC = 33
OPS_BWD_PAIR_EXEC = 38


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during a timed region: every 20 ms,
    and the region starts only once the first sample is in (nvidia-smi takes
    a while to start), so a region of a few hundred milliseconds still gets
    samples from inside it."""

    def __init__(self, index=0, tag="timed"):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gsr_bench_clocks_{tag}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
            self.skip = 0
            with open(self.path) as fh:
                self.skip = sum(1 for _ in fh)   # samples taken before the region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            # a region shorter than the sampling interval gets the sample that
            # closes it (taken within one interval of its end)
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 0.2 and self.proc.poll() is None:
                self.fh.flush()
                with open(self.path) as fh:
                    if sum(1 for _ in fh) > getattr(self, "skip", 0):
                        break
                time.sleep(0.005)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            return self._summary()
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass

    def _summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for n, line in enumerate(open(self.path)):
            if n < getattr(self, "skip", 0):
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device=None):
    """Largest value of x over all ranks (x itself on one rank); the device is
    the process group's (cuda for nccl, cpu for gloo)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws, device=None):
    """Sum of x over all ranks (x itself on one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def _view_block(scene, a, b):
    """The scene with views [a, b) only (the same Gaussians)."""
    from paper_2512_08498_gb300 import scenes as S
    return S.Scene(scene.name, scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
                   scene.sh_degree, scene.views[a:b], tile=scene.tile, bg=scene.bg, target_seed=scene.target_seed)


def build_workload(name, scale, seed_offset):
    from paper_2512_08498_gb300 import scenes
    fn = scenes.WORKLOADS[name]
    import inspect
    sig = inspect.signature(fn).parameters
    kw = {"seed": sig["seed"].default + seed_offset}
    if scale != 1.0:
        kw["n"] = max(1, int(round(sig["n"].default * scale)))
    return fn(**kw)


# ---------------------------------------------------------------------------
# oracle (CPU) arm
# ---------------------------------------------------------------------------

def _one_view(scene, v):
    from paper_2512_08498_gb300 import scenes as S
    return S.Scene(scene.name, scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
                   scene.sh_degree, [scene.views[v]], tile=scene.tile, bg=scene.bg, target_seed=scene.target_seed)


def oracle_rows(scene, view=0, y0=0, rows=None):
    """Time the CPU oracle on view `view`: its full preprocess (decision
    mirror + FP64 projection) and tile lists, then forward + backward (L1
    loss against the seeded target) over the full-width rows [y0, y0 + rows)
    (default: every row).  Returns (seconds of the preprocess and lists,
    seconds of the rows' fwd + bwd, rows, threads)."""
    import oracle
    one = _one_view(scene, view)
    v = one.views[0]
    rows = v.height - y0 if rows is None else min(rows, v.height - y0)
    t0 = time.perf_counter()
    o = oracle.Oracle(one)
    o.mirror()
    o.rec64()
    o.lists()
    t_pre = time.perf_counter() - t0
    blocks = [(0, 0, y0, v.width, rows)]
    t1 = time.perf_counter()
    ref = o.forward(blocks=blocks)
    tgt = one.targets()[0][:, y0:y0 + rows, :]
    d = [np.sign(ref["rgb"][0] - tgt) / (3.0 * v.width * v.height)]
    o.backward(d, blocks=blocks)
    return t_pre, time.perf_counter() - t1, rows, oracle.num_threads()


def oracle_full_view(scene, view=0):
    """One full view, end to end, timed (no extrapolation)."""
    t_pre, t_px, _, thr = oracle_rows(scene, view)
    v = scene.views[view]
    desc = (f"view {view} of {scene.name} in full: preprocess + tile lists ({t_pre:.2f} s) and fwd+bwd over all "
            f"{v.width}x{v.height} pixels ({t_px:.2f} s), timed end to end")
    return t_pre + t_px, desc, thr


def oracle_band(scene, view, band, n_bands):
    """View `view`'s preprocess and lists, and fwd+bwd over row band `band` of
    n_bands full-width bands; the view's time extrapolated as preprocess +
    n_bands x band."""
    v = scene.views[view]
    h = -(-v.height // n_bands)
    y0 = min(band * h, v.height - 1)
    t_pre, t_px, rows, thr = oracle_rows(scene, view, y0, h)
    per_view = t_pre + t_px * v.height / float(rows)
    desc = (f"view {view} of {scene.name}: preprocess + tile lists ({t_pre:.2f} s) and fwd+bwd over rows "
            f"{y0}..{y0 + rows - 1} of {v.height}, full width ({t_px:.2f} s), scaled to the view")
    return per_view, desc, thr


def bench_config(scene, args, ws=1):
    return {"workload": scene.name, "views": len(scene.views),
            "resolution": f"{scene.views[0].width}x{scene.views[0].height}",
            "gaussians": scene.n, "sh_degree": scene.sh_degree,
            "tile": list(args.tile), "blend_batch": args.batch,
            "blend_batch_bwd": args.batch_bwd,
            "l2": "inputs larger than L2 (Gaussian parameters alone exceed 129 MB)",
            "parallelism": ("1 GPU" if ws == 1 else
                            f"the batch's views sharded over {ws} ranks (Gaussians replicated), one all-reduce "
                            f"of the parameter gradients per step")}


REF_BANDS = 8


def run_reference(args):
    """The oracle on the machine's host cores.  Step i renders view
    (i // REF_BANDS) mod V: its full preprocess and tile lists, and fwd+bwd
    over full-width row band i mod REF_BANDS, scaled to the view; every
    REF_BANDS consecutive steps cover one view's full frame."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    scene = build_workload(args.workload, args.scale, 0)
    nv = len(scene.views)
    for i in range(args.warmup):
        oracle_band(scene, (i // REF_BANDS) % nv, i % REF_BANDS, REF_BANDS)
    times, thr = [], 1
    for i in range(args.steps):
        pv, _, thr = oracle_band(scene, (i // REF_BANDS) % nv, i % REF_BANDS, REF_BANDS)
        times.append(pv * nv)
    t = statistics.median(times)
    value = nv / t
    v = scene.views[0]
    desc = (f"per step: one view's full preprocess + tile lists and fwd+bwd over one of {REF_BANDS} full-width "
            f"row bands of its {v.width}x{v.height} frame, scaled to the view; the bands rotate, so every "
            f"{REF_BANDS} steps time one full frame; value = views / (median step time x {nv})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(scene, args, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2512_08498_gb300.rasterizer import Rasterizer, l1_loss_grad, to_camera_views
    from paper_2512_08498_gb300.sharding import GradBuffer, allreduce_grads, shard_bounds, shard_views

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    # every rank: the same Gaussians and views; rank r renders its block of the views
    full = build_workload(args.workload, args.scale, 0)
    v0, v1 = shard_views(full.views, rank, ws)
    n_views_total = len(full.views)
    scene = _view_block(full, v0, v1)
    n_views = len(scene.views)
    has_views = n_views > 0
    npix = sum(v.width * v.height for v in scene.views)
    K = (scene.sh_degree + 1) ** 2
    params = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
              (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh.reshape(scene.n, K, 3))]
    cams = to_camera_views(scene.views, dev)
    tg_views = full.targets()[v0:v1]
    tgt_host = torch.from_numpy(np.ascontiguousarray(np.concatenate([t.reshape(-1) for t in tg_views])
                                                     if tg_views else np.zeros(0, np.float32))).pin_memory()
    target = tgt_host.to(dev)

    r = Rasterizer(tile=tuple(args.tile), batch=args.batch, sh_degree=scene.sh_degree, bg=scene.bg, device=dev)
    r.set_config(batch_bwd=args.batch_bwd, list_prefix=args.list_prefix)
    rgb = torch.empty(3 * npix, device=dev)
    depth = torch.empty(npix, device=dev)
    alpha = torch.empty(npix, device=dev)
    dl = torch.empty_like(rgb)
    loss = torch.zeros(1, device=dev)
    # the parameter gradients in one flat buffer: one all-reduce per step
    gbuf = GradBuffer(scene.n, scene.sh_degree, dev)
    grads = gbuf.tensors() + (torch.empty(n_views, 6, device=dev),)
    saved = r.new_saved()
    stream = torch.cuda.current_stream(dev)

    def step(views=cams, sv=saved, out=(rgb, depth, alpha), dlb=dl, tg=target):
        if has_views:
            r.forward(params, views, saved=sv, out=out)
            l1_loss_grad(out[0], tg, dlb, loss)
            r.backward(params, views, sv, dlb, grads=grads)
        else:
            gbuf.flat.zero_()
        if ws > 1:
            allreduce_grads(gbuf)

    # the autotuner's tile shape and blend batches for this batch (timed
    # forward + backward of every supported choice), before anything is timed
    tuned = None
    if args.tune and has_views:
        l1_loss_grad(rgb, target, dl, loss)
        tuned = r.tune(params, cams, dl, saved=saved, out=(rgb, depth, alpha), grads=grads)
        args.tile, args.batch, args.batch_bwd = list(tuned["tile"]), tuned["batch"], tuned["batch_bwd"]

    # sizing call (synchronous), then the asynchronous steady state
    step()
    torch.cuda.synchronize(dev)
    info0 = saved.info() if has_views else None
    # the timed steps skip the forward's pair counters (statistics only); the
    # counts come from the sizing call above, on the same inputs
    r.set_config(no_sync=True, pair_counts=False)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- timed region (device time, CUDA events on the launching stream) ----
    # plain steps: the library's per-phase events (profile) stay off here and
    # are recorded in a second pass of the same steps below
    launches0 = r.stats()["launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms_total = e0.elapsed_time(e1)
    launches = r.stats()["launches"] - launches0
    if has_views:
        r.check(saved)
    # ---- per-phase device times: the same steps again, events between the phases ----
    r.set_config(profile=True)
    r.stats()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    st = r.stats()
    r.set_config(profile=False)
    ms_step = ms_total / args.steps
    ms_step = max_over_ranks(ms_step, ws, dev)
    info = saved.info()
    if info0 is not None:
        info.update({k: info0[k] for k in ("fwd_pairs", "blended_pairs")})
    pairs = sum_over_ranks(info["fwd_pairs"] + info["bwd_pairs"], ws, dev)
    # whole job: every view of the batch over the slowest rank's step
    value = n_views_total / (ms_step / 1000.0)

    # ---- the one exchange of a view-sharded step, timed alone ----
    allreduce = None
    if ws > 1:
        for _ in range(3):
            allreduce_grads(gbuf)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        barrier()
        a0.record(stream)
        for _ in range(args.steps):
            allreduce_grads(gbuf)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ar_ms = max_over_ranks(a0.elapsed_time(a1) / args.steps, ws, dev)
        nbytes = gbuf.flat.numel() * 4
        allreduce = {"ms": ar_ms, "bytes": nbytes, "algbw_gbs": nbytes / (ar_ms * 1e-3) / 1e9,
                     "views_per_rank": [b - a for a, b in zip(shard_bounds(
                         [v.width * v.height for v in full.views], ws)[:-1], shard_bounds(
                         [v.width * v.height for v in full.views], ws)[1:])]}

    # ---- end to end through the public API with host buffers ----
    # (right after the device-timed region, before the other measurements)
    e2e = None
    if not args.no_e2e:
        with ClockSampler(dev.index, "e2e") as clk_e2e:
            e2e = run_e2e(args, r, step, target, tgt_host, grads, loss, saved, n_views, n_views_total, ws, dev,
                          has_views)
        e2e["clocks"] = clk_e2e.summary()

    # ---- the same step replayed from one CUDA graph ----
    # forward, loss and backward captured once (the library enqueues no host
    # synchronisation under GSR_FLAG_NO_SYNC); K replays timed with CUDA
    # events on the replaying stream
    graph_step = None
    if not args.no_graph and ws == 1:
        r.set_config(no_sync=True)
        gstream = torch.cuda.Stream(dev)
        gstream.wait_stream(stream)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gstream):
            with torch.cuda.graph(cg, stream=gstream):
                step()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(gstream):
            for _ in range(max(args.warmup, 3)):
                cg.replay()
            torch.cuda.synchronize(dev)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            g0.record(gstream)
            for _ in range(args.steps):
                cg.replay()
            g1.record(gstream)
        torch.cuda.synchronize(dev)
        barrier()
        r.check(saved)
        g_ms = max_over_ranks(g0.elapsed_time(g1) / args.steps, ws, dev)
        graph_step = {"value": n_views_total / (g_ms / 1000.0), "unit": UNIT, "ms_per_step": g_ms,
                      "speedup_vs_eager": ms_step / g_ms}
        del cg

    # ---- roofline per phase, and of the whole step ----
    # Each phase's algorithmic work (bytes for the data-movement phases, useful
    # FP32 operations for the blends) over its live CUDA-event time, against
    # the measured copy bandwidth or the FP32 ALU roof; the step's fraction is
    # the sum of the phases' roof times over the measured step time.
    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    phase = {k: v / max(1, st["calls"][k]) for k, v in st["phase_ms"].items()}
    dom = max(phase, key=phase.get)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * sm_max * 1e6 / 1e12   # T FP32 ops/s
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    M, NV, MF = info["n_instances"], info["n_visible"], info["n_instances_full"]
    tile_passes = (max(1, math.ceil(math.log2(max(2, info["n_tiles"])))) + 7) // 8
    row_bytes = 12 + 12 + 16 + 4 + 12 * K          # one Gaussian's parameters (= its gradient row)
    param_bytes = scene.n * row_bytes
    rows = info["grad_rows"]                        # Gaussians with a visible record (per view group)
    work = {
        "preprocess": ("hbm", param_bytes + NV * (64 + 4 + 16)),
        "depth_sort": ("hbm", NV * 4 * 20),
        # each visible record's inputs read once (sorted id, aux, mean/conic/opacity: 52 B),
        # each kept (tile, record) pair written once
        "duplicate": ("hbm", NV * (4 + 16 + 32) + M * 8),
        "tile_sort": ("hbm", M * tile_passes * 20),
        "ranges": ("hbm", M * 4 + info["n_tiles"] * 8),
        "blend_fwd": ("alu", info["blended_pairs"] * OPS_FWD_PAIR),
        # the per-record gradient clear; the parameter gradients are cleared on
        # a side stream while the backward blend runs, outside this phase
        "bwd_clear": ("hbm", NV * 48),
        "blend_bwd": ("alu", info["blended_pairs"] * OPS_BWD_PAIR),
        # per visible record its gradient (48 B) and aux (16 B) read; per touched
        # Gaussian its parameters read and its gradient row written, once
        "preprocess_bwd": ("hbm", NV * (48 + 16) + 2 * rows * row_bytes),
    }
    exec_ops = {"blend_fwd": OPS_FWD_PAIR_EXEC, "blend_bwd": OPS_BWD_PAIR_EXEC}
    phases = {}
    roof_ms = 0.0
    for k, (bound, amount) in work.items():
        if k not in phase or phase[k] <= 0:
            continue
        if bound == "alu":
            ach, peak, unit = amount / (phase[k] * 1e-3) / 1e12, alu_peak, "TFLOP/s"
            t_roof = amount / (alu_peak * 1e12) * 1e3
        else:
            ach, peak, unit = amount / (phase[k] * 1e-3) / 1e9, hbm, "GB/s"
            t_roof = amount / (hbm * 1e9) * 1e3
        roof_ms += t_roof
        phases[k] = {"bound": bound, "ms": phase[k], "roof_ms": t_roof, "achieved": ach, "peak": peak,
                     "unit": unit, "frac": ach / peak}
        if k in exec_ops:
            # the same pairs at the operations the kernel executes per pair
            ops = OPS_FWD_PAIR if k == "blend_fwd" else OPS_BWD_PAIR
            phases[k]["ops_per_pair"] = ops
            phases[k]["ops_per_pair_executed"] = exec_ops[k]
            phases[k]["frac_executed"] = ach / peak * exec_ops[k] / ops
    profiled = (args.workload, args.scale, tuple(args.tile), args.batch, args.batch_bwd) == PROFILED_CONFIG
    if dom not in phases:   # a rank without views (more ranks than views)
        phases[dom] = {"bound": "hbm", "ms": 0.0, "roof_ms": 0.0, "achieved": 0.0, "peak": hbm, "unit": "GB/s",
                       "frac": 0.0}
    roof = dict(phases[dom])
    roof.pop("ms"); roof.pop("roof_ms")
    roof["traffic"] = PROFILED_DRAM_BYTES.get(dom) if profiled else None
    roof["kernel"] = dom
    roof["peak_source"] = (f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({peak_kind} max clock)"
                           if roof["bound"] == "alu" else f"{peak_kind} copy bandwidth")
    roof_total = {"roof_ms": roof_ms, "measured_ms": ms_step, "frac": roof_ms / ms_step,
                  "rank": rank if ws > 1 else None}

    # ---- next row: insertion probability and scale initialisation (Sec. 3.2) ----
    # run once per keyframe on the rendered views (not part of the
    # optimisation step); timed alone, device-resident inputs
    insertion = None
    if not args.no_insertion and ws == 1:
        r.set_config(no_sync=True)
        dist = (depth / alpha.clamp_min(1e-3)).clamp_min(0.2)
        ins_out = (torch.empty(npix, device=dev), torch.empty(npix, device=dev),
                   torch.empty(npix, dtype=torch.int32, device=dev))
        for _ in range(3):
            r.insertion(target, rgb, dist, cams, out=ins_out, read_count=False)
        reps = max(args.steps, 5)
        i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        i0.record(stream)
        for _ in range(reps):
            _, _, _, cnt = r.insertion(target, rgb, dist, cams, out=ins_out, read_count=False)
        i1.record(stream)
        torch.cuda.synchronize(dev)
        ins_ms = i0.elapsed_time(i1) / reps
        n_ins = int(cnt.item())
        ins_bytes = npix * (3 * 4 * 2 + 4 + 4 + 4) + npix * 4 + n_ins * 4
        insertion = {"ms": ins_ms, "views_per_s": n_views / (ins_ms * 1e-3), "inserted": n_ins,
                     "roofline": {"bound": "hbm", "achieved": ins_bytes / (ins_ms * 1e-3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": ins_bytes / (ins_ms * 1e-3) / 1e9 / hbm},
                     "sigma": 1.0, "tau_a": 0.2}

    # ---- next row: inter-camera merging (Sec. 3.2, Eq. 7-8) ----
    # each camera's samples (the insertion above) merged with the 1M scene
    # Gaussians as the existing set; one merge per camera, timed alone
    merging = None
    if not args.no_merging and insertion is not None:
        idx_all = ins_out[2][: insertion["inserted"]].cpu().numpy().view(np.uint32).astype(np.int64)
        offs = np.cumsum([0] + [v.width * v.height for v in scene.views])
        jobs = []
        for i, v in enumerate(scene.views):
            a, b = int(offs[i]), int(offs[i + 1])
            loc = idx_all[(idx_all >= a) & (idx_all < b)] - a
            jobs.append((cams[i], torch.from_numpy(loc.astype(np.int32)).to(dev), ins_out[1][a:b], dist[a:b],
                         target[3 * a:3 * b]))

        def merge_all():
            outs = []
            for cam_i, pix_i, sc_i, d_i, g_i in jobs:
                outs.append(r.merge(cam_i, params[0], params[1], params[4], pix_i, sc_i, d_i, g_i, tau_d=0.5))
            return outs
        for _ in range(3):
            merge_all()
        torch.cuda.synchronize(dev)
        # the six merges replayed from one CUDA graph (no launch gaps); eager if capture fails
        graph = None
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                g_outs = merge_all()
            graph.replay()
            torch.cuda.synchronize(dev)
        except Exception:   # pragma: no cover - capture unavailable
            graph = None
        reps = max(args.steps, 5)
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        m0.record(stream)
        for _ in range(reps):
            if graph is not None:
                graph.replay()
            else:
                g_outs = merge_all()
        m1.record(stream)
        torch.cuda.synchronize(dev)
        m_ms = m0.elapsed_time(m1) / reps
        mouts = g_outs
        n_samp = sum(int(j[1].numel()) for j in jobs)
        acts = torch.cat([o["sample_action"] for o in mouts]).cpu().numpy()
        kept_ex = sum(int((o["existing_action"] == 2).sum().item()) for o in mouts)
        # per camera: 24 B per existing Gaussian (mean, pair index written and
        # read, action), 4 B per pixel (slot map), 124 B per sample
        m_bytes = n_views * scene.n * 24 + npix * 4 + n_samp * 124
        merging = {"ms": m_ms, "cameras": n_views, "existing": scene.n, "samples": n_samp,
                   "inserted": int((acts == 0).sum()), "merged": int((acts == 1).sum()),
                   "replaced": int((acts == 2).sum()), "existing_kept": kept_ex, "tau_d": 0.5,
                   "cuda_graph": graph is not None,
                   "roofline": {"bound": "hbm", "achieved": m_bytes / (m_ms * 1e-3) / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": m_bytes / (m_ms * 1e-3) / 1e9 / hbm, "bytes": m_bytes}}

    # ---- next row: frequency-based scheduling (Sec. 3.3, Eq. 9-12) ----
    # X of the ground truth, of the ground truth at level 2 and of the
    # renderings for every view, then r, r', level-up and 1024 sampled frames;
    # timed alone, device-resident inputs
    frequency = None
    if not args.no_frequency and ws == 1:
        imgs = []
        o = 0
        for v in scene.views:
            n3 = 3 * v.width * v.height
            imgs.append((target[o:o + n3], v.width, v.height))
            o += n3
        o = 0
        rens = []
        for v in scene.views:
            n3 = 3 * v.width * v.height
            rens.append((rgb[o:o + n3], v.width, v.height))
            o += n3
        batch = [(t, w, h, 1) for t, w, h in imgs] + [(t, w, h, 2) for t, w, h in imgs] + [(t, w, h, 1) for t, w, h in rens]
        xs = torch.empty(len(batch), device=dev)
        uni = torch.rand(1024, device=dev, generator=torch.Generator(device=dev).manual_seed(5))

        def sched():
            r.dft_energy(batch, out=xs)
            return r.frequency_schedule(xs[:n_views], xs[2 * n_views:], x_gt_level=xs[n_views:2 * n_views],
                                        tau_f=2.0, uniforms=uni)
        for _ in range(3):
            sched()
        reps = max(args.steps, 5)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        f0.record(stream)
        for _ in range(reps):
            sres = sched()
        f1.record(stream)
        torch.cuda.synchronize(dev)
        f_ms = f0.elapsed_time(f1) / reps
        f_bytes = 0
        for t, w, h, fac in batch:
            wd, hd = w // fac, h // fac
            f_bytes += 12 * (wd * fac) * (hd * fac) + 2 * 3 * hd * (wd // 2 + 1) * 8
        frequency = {"ms": f_ms, "images": len(batch), "views_per_s": n_views / (f_ms * 1e-3),
                     "levels_up": int(sres["level_up"].sum().item()),
                     "roofline": {"bound": "hbm", "achieved": f_bytes / (f_ms * 1e-3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": f_bytes / (f_ms * 1e-3) / 1e9 / hbm,
                                  "bytes": f_bytes},
                     "tau_f": 2.0}

    # ---- the same batch as sequential single-view calls ----
    per_view = None
    if not args.no_per_view and ws == 1:
        singles = []
        offs = [0]
        for v in scene.views:
            offs.append(offs[-1] + v.width * v.height)
        for i in range(n_views):
            a, b = offs[i], offs[i + 1]
            sv = r.new_saved()
            singles.append((cams[i:i + 1], sv, (rgb[3 * a:3 * b], depth[a:b], alpha[a:b]), dl[3 * a:3 * b],
                            target[3 * a:3 * b]))
        r.set_config(no_sync=False)
        for (vv, sv, out, dlb, tg) in singles:
            step(vv, sv, out, dlb, tg)
        r.set_config(no_sync=True)
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            for (vv, sv, out, dlb, tg) in singles:
                step(vv, sv, out, dlb, tg)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        pv_ms = f0.elapsed_time(f1) / args.steps
        for (_, sv, _, _, _) in singles:
            r.check(sv)
        per_view = {"value": n_views / (pv_ms / 1000.0), "unit": UNIT, "ms_per_step": pv_ms,
                    "speedup_batched": pv_ms / ms_step}

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    # one full view end to end on all host cores; on one core, a band of rows
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        per_view_s, desc, thr = oracle_full_view(scene, 0)
        cpu = {"value": 1.0 / per_view_s, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc}
        oracle.set_num_threads(1)
        try:
            pv1, desc1, _ = oracle_band(scene, 0, REF_BANDS // 2, 4 * REF_BANDS)
        finally:
            oracle.set_num_threads(thr)
        cpu["value_1core"] = 1.0 / pv1
        cpu["sample_1core"] = desc1

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(full, args, ws),
            "allreduce": allreduce,
            "gaussian_pixel_pairs_per_s": pairs / (ms_step / 1000.0),
            "per_view": per_view,
            "graph": graph_step,
            "roofline": roof,
            "roofline_phases": phases,
            "roofline_total": roof_total,
            "phase_ms": phase,
            "counts": {"visible_records": NV, "instances": M, "grad_rows": rows, "fwd_pairs": info["fwd_pairs"],
                       "bwd_pairs": info["bwd_pairs"], "blended_pairs": info["blended_pairs"],
                       "warp_entries_fwd": info["warp_entries_fwd"], "warp_entries_bwd": info["warp_entries_bwd"],
                       "instances_full": MF,
                       "first_call_instances": info0["n_instances"] if info0 else 0,
                       "list_prefix": info["list_prefix"], "open_tiles": info["open_tiles"],
                       "instances_second_round": info["n_instances_second"]},
            "insertion": insertion,
            "merging": merging,
            "frequency": frequency,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_e2e(args, r, step, target, tgt_host, grads, loss, saved, n_views, n_views_total, ws, dev, has_views=True):
    """Same step through the public API with host buffers: every step's target
    images go host -> device and its loss and pose gradients come back, all
    inside the timed region.  The copies are pipelined as a training loop
    would: two device target buffers alternate; once step i's results are read
    back, step i + 2's targets stream into step i's buffer on a copy stream
    while step i + 1 runs, and the host waits for step i - 1's results (not
    step i's) before it enqueues step i + 1."""
    import torch
    h2d = tgt_host.numel() * 4
    pose_host = [torch.empty(n_views, 6).pin_memory() for _ in range(2)]
    loss_host = [torch.empty(1).pin_memory() for _ in range(2)]
    d2h = (pose_host[0].numel() + loss_host[0].numel()) * 4
    bufs = [target, torch.empty_like(target)]
    comp = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    results = [torch.cuda.Event() for _ in range(2)]
    r.set_config(no_sync=True)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    K = args.steps
    t0 = time.perf_counter()
    with torch.cuda.stream(copy):
        for j in range(min(2, K)):
            bufs[j].copy_(tgt_host, non_blocking=True)
            copied[j].record(copy)
    for i in range(K):
        b = i & 1
        comp.wait_event(copied[b])
        step(tg=bufs[b])
        pose_host[b].copy_(grads[5], non_blocking=True)
        loss_host[b].copy_(loss, non_blocking=True)
        results[b].record(comp)
        if i + 2 < K:
            # after the small read-back, not just after the step: a large
            # upload that takes the copy engine first would hold the read-back,
            # and the next step behind it in stream order
            copy.wait_event(results[b])
            with torch.cuda.stream(copy):
                bufs[b].copy_(tgt_host, non_blocking=True)
                copied[b].record(copy)
        if i >= 1:
            results[b ^ 1].synchronize()   # step i - 1's loss and pose gradients are on the host
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / K, ws, dev)
    if has_views:
        r.check(saved)
    return {"value": n_views_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000.0 * e2e_s, "pipelined": True}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rig6")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--tile", type=int, nargs=2, default=[16, 16])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--batch-bwd", type=int, default=128, help="backward blend batch")
    ap.add_argument("--list-prefix", type=float, default=0.0,
                    help="tile lists: 0 two rounds with the automatic first-round fraction (default), "
                         "f in (0, 1) that fraction, >= 1 one round")
    ap.add_argument("--no-per-view", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-insertion", action="store_true")
    ap.add_argument("--no-frequency", action="store_true")
    ap.add_argument("--no-merging", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--tune", action="store_true", help="use the autotuner's tile shape and blend batches")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
