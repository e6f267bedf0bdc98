"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded scene and compare.

Bars: sort keys, values, tile ranges, per-record binary32 projections and
per-pixel contributor counts bit-exact; RGB and alpha within 2e-5 max-abs,
depth within 2e-5 relative (max-abs / max(1, |depth|)); gradients within 1e-4
relative L2 of the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views

IMG_TOL = 2e-5
GRAD_TOL = 1e-4
PARAM_NAMES = ["means", "log_scales", "quats", "opacity_logits", "sh"]


def device():
    return torch.device("cuda", 0)


def params_of(scene, dev=None):
    dev = dev or device()
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in
            (scene.means, scene.log_scales, scene.quats, scene.opacity_logits,
             scene.sh.reshape(scene.n, (scene.sh_degree + 1) ** 2, 3))]


def upstream(scene, o: oracle.Oracle, ref, seed=0, depth_w=0.05, alpha_w=0.3):
    """L1-style upstream gradient from the oracle's image (never from the GPU) plus
    seeded depth/alpha gradients.  Returns per-view lists (for the oracle) and flat
    float32 arrays (for the GPU)."""
    rng = np.random.default_rng(seed)
    targets = scene.targets()
    d_rgb, d_dep, d_alp = [], [], []
    for i, v in enumerate(scene.views):
        n = 3 * v.width * v.height
        d_rgb.append((np.sign(ref["rgb"][i] - targets[i]) / n).astype(np.float32).astype(np.float64))
        d_dep.append((depth_w * rng.standard_normal((v.height, v.width)) / n).astype(np.float32).astype(np.float64))
        d_alp.append((alpha_w * rng.standard_normal((v.height, v.width)) / n).astype(np.float32).astype(np.float64))
    flat = lambda xs: np.ascontiguousarray(np.concatenate([x.reshape(-1) for x in xs]).astype(np.float32))
    return (d_rgb, d_dep, d_alp), (flat(d_rgb), flat(d_dep), flat(d_alp))


def run_gpu(scene, tile=None, batch=256, grads=None, raster=None, batch_bwd=None):
    dev = device()
    tile = tile or scene.tile
    r = raster or Rasterizer(tile=tile, batch=batch, sh_degree=scene.sh_degree, bg=scene.bg, device=dev)
    if batch_bwd is not None:
        r.set_config(batch_bwd=batch_bwd)
    params = params_of(scene, dev)
    cams = to_camera_views(scene.views, dev)
    rgb, depth, alpha, saved = r.forward(params, cams)
    keys, vals, ranges = r.debug_lists(saved)
    rec, rect, flags = r.debug_records(saved)
    tf, nc = r.debug_pixels(saved)
    out = dict(rgb=rgb.cpu().numpy(), depth=depth.cpu().numpy(), alpha=alpha.cpu().numpy(),
               keys=keys.cpu().numpy().view(np.uint64), vals=vals.cpu().numpy().view(np.uint32),
               ranges=ranges.cpu().numpy().view(np.uint32), rec=rec.cpu().numpy(), rect=rect.cpu().numpy(),
               flags=flags.cpu().numpy().view(np.uint32), tfinal=tf.cpu().numpy(),
               ncontrib=nc.cpu().numpy().view(np.uint32), info=saved.info())
    if grads is not None:
        d_rgb, d_dep, d_alp = (torch.from_numpy(x).to(dev) for x in grads)
        g = r.backward(params, cams, saved, d_rgb, d_dep, d_alp, want_focal=True)
        out["grads"] = {n: t.cpu().numpy().astype(np.float64) for n, t in zip(PARAM_NAMES, g[:5])}
        out["grads"]["pose"] = g[5].cpu().numpy().astype(np.float64)
        out["grads"]["focal"] = g[6].cpu().numpy().astype(np.float64)
        out["grec"] = r.debug_record_grads(saved).cpu().numpy()
        out["info"] = saved.info()
    out["raster"] = r
    return out


def flat_views(xs):
    return np.concatenate([np.asarray(x).reshape(-1) for x in xs])


def compare_lists(g, o: oracle.Oracle):
    keys, vals, ranges = o.lists()
    assert g["keys"].shape == keys.shape, (g["keys"].shape, keys.shape)
    assert np.array_equal(g["keys"], keys), "sort keys differ"
    assert np.array_equal(g["vals"], vals), "sort values (record indices) differ"
    assert np.array_equal(g["ranges"], ranges), "tile ranges differ"


def compare_records(g, o: oracle.Oracle):
    m = o.mirror()
    culled = (m["flags"] & 1) != 0
    assert np.array_equal((g["flags"] & 1) != 0, culled), "cull decisions differ"
    vis = ~culled
    rec = g["rec"][vis]
    bl = m["blend"][vis]
    # u, v, qa, qb, qc, sigma: bit-exact binary32
    for j, col in enumerate([0, 1, 2, 3, 4, 5]):
        assert np.array_equal(rec[:, col].view(np.uint32), bl[:, j].view(np.uint32)), f"record field {j} differs"
    assert np.array_equal(rec[:, 6].view(np.uint32), m["zbits"][vis]), "depth bits differ"
    assert np.array_equal(rec[:, 8:11].view(np.uint32), m["colour"][vis].view(np.uint32)), "colour differs"
    assert np.array_equal(g["rect"][vis], m["rect"][vis]), "tile rectangles differ"


def compare_pixels(g, ref):
    nc = flat_views(ref["ncontrib"]).astype(np.uint32)
    bad = np.nonzero(g["ncontrib"] != nc)[0]
    assert bad.size == 0, f"{bad.size} contributor counts differ, first at {bad[:5]}"
    tf = flat_views(ref["tfinal"])
    assert np.abs(g["tfinal"] - tf).max() <= IMG_TOL


def compare_counters(g, ref, with_bwd: bool):
    """The throughput counters (examined pairs, contributor sum, composited
    pairs) equal the oracle's per-pixel counts summed."""
    info = g["info"]
    assert info["fwd_pairs"] == int(flat_views(ref["nexam"]).astype(np.int64).sum())
    assert info["blended_pairs"] == int(flat_views(ref["nblend"]).astype(np.int64).sum())
    if with_bwd:
        assert info["bwd_pairs"] == int(flat_views(ref["ncontrib"]).astype(np.int64).sum())


def compare_images(g, ref):
    rgb = flat_views(ref["rgb"])
    err = np.abs(g["rgb"] - rgb).max() if rgb.size else 0.0
    assert err <= IMG_TOL, f"rgb max-abs {err}"
    alpha = flat_views(ref["alpha"])
    err_a = np.abs(g["alpha"] - alpha).max() if alpha.size else 0.0
    assert err_a <= IMG_TOL, f"alpha max-abs {err_a}"
    dep = flat_views(ref["depth"])
    err_d = (np.abs(g["depth"] - dep) / np.maximum(1.0, np.abs(dep))).max() if dep.size else 0.0
    assert err_d <= IMG_TOL, f"depth rel {err_d}"
    return err, err_a, err_d


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def compare_grads(g, go, tol=GRAD_TOL):
    errs = {}
    for name in PARAM_NAMES + ["pose", "focal"]:
        e = rel_l2(g["grads"][name], go[name])
        errs[name] = e
        assert e <= tol, f"grad {name}: rel L2 {e:.3e} > {tol}"
    return errs
