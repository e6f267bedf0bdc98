"""Writes the stored oracle values under tests/golden/ (regression fixtures).

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``paper_2512_08498_gb300.scenes``, which hold none of the method's
arithmetic).  The paper prints no rasterizer, insertion, merging or scheduler
output, so these values are not the paper's: they freeze what the pinned
oracle computes, so that any later change to its arithmetic shows up as a
failing ``tests/test_oracle_golden.py`` and has to be regenerated here, with
the passage (or the reading of it) that justifies the change named in the
commit.

Usage (from the repository root):  python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FIXTURE = os.path.join(HERE, "oracle_values.txt")


def _sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def _scene_digest(s) -> str:
    parts = [s.means, s.log_scales, s.quats, s.opacity_logits, s.sh]
    for v in s.views:
        parts.append(np.array([v.width, v.height, v.fx, v.fy, v.cx, v.cy], np.float64))
        parts.append(np.asarray(v.viewmat, np.float32))
        if v.subset is not None:
            parts.append(np.asarray(v.subset, np.uint32))
    parts += s.targets()
    return _sha(*parts)


def _raster(name: str, scene, tile=None) -> dict:
    """Lists, forward and the adjoint of the mean L1 loss against the scene's
    seeded targets (dL/drgb = sign(C - T) / (3 H W) per view)."""
    import oracle

    o = oracle.Oracle(scene, tile=tile)
    keys, vals, ranges = o.lists()
    f = o.forward()
    tg = scene.targets()
    dl = [np.sign(f["rgb"][i] - tg[i].astype(np.float64)) / tg[i].size for i in range(len(tg))]
    g = o.backward(dl)
    out = {
        f"{name}.inputs_sha256": _scene_digest(scene),
        f"{name}.instances": int(keys.shape[0]),
        f"{name}.keys_sha256": _sha(keys.astype(np.uint64)),
        f"{name}.vals_sha256": _sha(vals.astype(np.uint32)),
        f"{name}.ranges_sha256": _sha(ranges.astype(np.uint32)),
        f"{name}.ncontrib_sha256": _sha(*[x.astype(np.uint32) for x in f["ncontrib"]]),
        f"{name}.nexam_sha256": _sha(*[x.astype(np.uint32) for x in f["nexam"]]),
        f"{name}.ncontrib_sum": int(sum(int(x.sum()) for x in f["ncontrib"])),
        f"{name}.nblend_sum": int(sum(int(x.sum()) for x in f["nblend"])),
        f"{name}.stoprec_sha256": _sha(*[x.astype(np.uint32) for x in f["stoprec"]]),
        f"{name}.reach_count": int(o.reach().astype(np.int64).sum()),
    }
    for key in ("rgb", "depth", "alpha", "tfinal"):
        out[f"{name}.{key}_sum"] = float(sum(float(x.sum()) for x in f[key]))
        out[f"{name}.{key}_sumsq"] = float(sum(float((x * x).sum()) for x in f[key]))
    out[f"{name}.loss_l1"] = float(sum(float(np.abs(f["rgb"][i] - tg[i]).mean()) for i in range(len(tg))))
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose", "focal"):
        a = np.asarray(g[key], np.float64)
        out[f"{name}.grad_{key}_norm"] = float(np.linalg.norm(a))
        out[f"{name}.grad_{key}_sum"] = float(a.sum())
    # full rows of the three Gaussians with the largest mean gradient
    gm = np.linalg.norm(np.asarray(g["means"]).reshape(scene.n, 3), axis=1)
    for r, j in enumerate(np.argsort(-gm, kind="stable")[:3]):
        out[f"{name}.top{r}_index"] = int(j)
        for key in ("means", "log_scales", "quats", "opacity_logits"):
            row = np.atleast_1d(np.asarray(g[key])[j]).reshape(-1)
            for c, v in enumerate(row):
                out[f"{name}.top{r}_{key}_{c}"] = float(v)
    return out


def compute() -> dict:
    """Every stored value, recomputed from the oracle."""
    import oracle
    from oracle import frequency, merging
    from paper_2512_08498_gb300 import scenes

    oracle.build()
    out = {}
    # 10k Gaussians, one 256 x 256 view, SH 0, 16 x 16 tiles
    small = scenes.small_box()
    out.update(_raster("small_box", small))
    # three views of mixed sizes, ascending subsets, SH 2, 32 x 8 tiles, grey background
    views = [scenes.pinhole(96, 64, f=80.0),
             scenes.pinhole(50, 70, f=60.0, viewmat=scenes.look_from([0.3, -0.1, -0.5], yaw_deg=8.0),
                            subset=np.arange(0, 3000, 2, dtype=np.uint32)),
             scenes.pinhole(33, 17, f=30.0, viewmat=scenes.look_from([-0.2, 0.1, 0.2], yaw_deg=-5.0, roll_deg=3.0),
                            subset=np.arange(500, 2600, dtype=np.uint32))]
    multi = scenes.random_scene(7, 3000, views, 2, tile=(32, 8), bg=(0.1, 0.2, 0.3))
    out.update(_raster("multi_view", multi))

    # insertion (Eq. 4-6) on the small view: ground truth = the seeded target,
    # rendered = the oracle's own render, depth = its depth over alpha
    o = oracle.Oracle(small)
    f = o.forward()
    rgb = f["rgb"][0].astype(np.float32)
    a = f["alpha"][0]
    depth = np.where(a > 0, f["depth"][0] / np.maximum(a, 1e-30), 0.0).astype(np.float32)
    gt = small.targets()[0]
    ins = oracle.insertion(gt, rgb, depth, small.views[0].fx, sigma=1.0, tau_a=0.2)
    out["insertion.inserted"] = int(ins["inserted"].sum())
    out["insertion.inserted_sha256"] = _sha(ins["inserted"].astype(np.uint8))
    for key in ("p_gt", "p_ren", "p_a", "scale"):
        out[f"insertion.{key}_sum"] = float(ins[key].sum())

    # merging (Eq. 7-8): the small scene's Gaussians reprojected into its view
    # against the samples just chosen
    pix = np.nonzero(ins["inserted"].reshape(-1))[0].astype(np.int64)
    dc = np.asarray(small.sh, np.float64).reshape(small.n, -1, 3)[:, 0, :]
    m = merging.merge(small.views[0], small.means, small.log_scales, dc, pix, ins["scale"].astype(np.float32),
                      depth, gt, tau_d=0.5)
    out["merging.samples"] = int(pix.shape[0])
    for key in ("pair", "sample_action", "existing_action"):
        out[f"merging.{key}_sha256"] = _sha(np.asarray(m[key]).astype(np.int64))
    for key in ("sample_dc", "sample_depth", "sample_scale", "existing_dc"):
        out[f"merging.{key}_sum"] = float(np.asarray(m[key], np.float64).sum())

    # frequency energy (Eq. 10) and the scheduler (Eq. 9, 12)
    tg = multi.targets()
    xs = [frequency.dft_energy(t) for t in tg]
    xl = [frequency.dft_energy(t, 2) for t in tg]
    xr = [frequency.dft_energy(np.sqrt(t)) for t in tg]
    for i in range(len(tg)):
        out[f"frequency.x_{i}"] = float(xs[i])
        out[f"frequency.x_level2_{i}"] = float(xl[i])
        out[f"frequency.x_sqrt_{i}"] = float(xr[i])
    u = np.random.default_rng(11).random(16).astype(np.float32)
    sch = frequency.frequency_schedule(xs, xl, xr, 2.0, u)
    out["frequency.samples"] = " ".join(str(int(v)) for v in sch["samples"])
    out["frequency.level_up"] = " ".join(str(int(v)) for v in sch["level_up"])
    return out


def write(values: dict, path: str = FIXTURE) -> None:
    with open(path, "w") as fh:
        fh.write("# Oracle regression values, written by tests/golden/make_golden.py (calls oracle/ only).\n")
        fh.write("# Not numbers printed by the paper: it prints none for these steps.\n")
        for k in sorted(values):
            v = values[k]
            fh.write(f"{k} = {v!r}\n" if isinstance(v, float) else f"{k} = {v}\n")


def read(path: str = FIXTURE) -> dict:
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(" = ", 1)
            out[k] = v
    return out


if __name__ == "__main__":
    write(compute())
    print(f"wrote {FIXTURE}")
