"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded scene and compare.

Bars: per-record binary32 projections bit-exact; RGB and alpha within 2e-5
max-abs, depth within 2e-5 relative (max-abs / max(1, |depth|)); gradients
within 1e-4 relative L2 of the FP64 oracle.

The oracle's tile lists are the plain ones: every non-culled record in every
tile of its rectangle.  The GPU lists fewer records per tile (it drops a record
from a tile when no pixel centre of the tile can reach alpha 1/255), so its
lists are one of several correct answers and are checked for what makes them
correct, exactly:
  * each GPU list is an ordered subsequence of the oracle's list of its tile
    (keys carry the record's depth bits; ranges partition the GPU's keys);
  * every entry of the oracle's lists that reaches alpha >= 1/255 at some
    in-view pixel centre of its tile (``Oracle.reach``) is kept;
  * per pixel, the record at the GPU's contributor count (the last composited
    record) is the oracle's, and the entry that stopped the pixel is kept;
  * the composited pair count is the oracle's, the examined count follows
    from the stop records.
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


def _pairs(keys, vals):
    """(tile << 32 | record) of each list entry: unique per list."""
    return ((keys >> np.uint64(32)) << np.uint64(32)) | vals.astype(np.uint64)


def _select_tiles(keys, vals, ranges, tiles):
    idx = np.concatenate([np.arange(ranges[t, 0], ranges[t, 1], dtype=np.int64) for t in tiles]) \
        if len(tiles) else np.zeros(0, np.int64)
    return keys[idx], vals[idx]


def compare_lists(g, o: oracle.Oracle, tiles=None, check_reach=True):
    """GPU lists vs the oracle's plain lists (see the module docstring).
    tiles: global tile ids to compare (the oracle restricted to them), or None
    for every tile."""
    okeys, ovals, oranges = o.lists()
    gk, gv, gr = g["keys"], g["vals"], g["ranges"].reshape(-1, 2)
    m = o.mirror()
    assert gk.shape == gv.shape
    # sorted by (tile, depth bits, record index), depth bits from the record
    if gk.size > 1:
        inc = (gk[1:] > gk[:-1]) | ((gk[1:] == gk[:-1]) & (gv[1:] > gv[:-1]))
        assert inc.all(), "GPU lists not sorted by (tile, depth, index)"
    assert np.array_equal((gk & np.uint64(0xFFFFFFFF)).astype(np.uint32), m["zbits"][gv]), "key depth bits differ"
    # ranges partition the keys by tile
    gt = (gk >> np.uint64(32)).astype(np.int64)
    t_all = np.arange(gr.shape[0])
    st, en = np.searchsorted(gt, t_all, "left"), np.searchsorted(gt, t_all, "right")
    exp = np.where((en > st)[:, None], np.stack([st, en], 1), 0)
    assert np.array_equal(gr.astype(np.int64), exp), "tile ranges do not partition the keys"
    if tiles is not None:
        gk, gv = _select_tiles(gk, gv, gr, sorted(tiles))
    else:
        assert g["info"]["n_instances_full"] == okeys.size, "rectangle instance count differs"
    gp, op = _pairs(gk, gv), _pairs(okeys, ovals)
    ops = np.sort(op)
    pos = np.searchsorted(ops, gp)
    ok = (pos < ops.size) & (ops[np.minimum(pos, max(ops.size - 1, 0))] == gp) if ops.size else gp.size == 0
    assert np.all(ok), f"{int(np.size(ok) - np.sum(ok))} GPU entries are in no oracle list"
    # ordered subsequence: both sorted by the same order and every entry known,
    # so only the kept set is left to check
    if check_reach:
        need = op[o.reach().astype(bool)]
        gps = np.sort(gp)
        p2 = np.searchsorted(gps, need)
        kept = (p2 < gps.size) & (gps[np.minimum(p2, max(gps.size - 1, 0))] == need) if gps.size else need.size == 0
        assert np.all(kept), f"{int(np.size(kept) - np.sum(kept))} entries reaching 1/255 were dropped"


def pixel_tiles(o: oracle.Oracle, blocks=None):
    """Global tile id of every pixel of ``blocks`` (default: the full views),
    flattened block after block in row-major order."""
    blocks = o.full_blocks() if blocks is None else blocks
    out = []
    tw, th = o.tile
    for (v, x0, y0, w, h) in blocks:
        ys, xs = np.mgrid[y0:y0 + h, x0:x0 + w]
        out.append((o.tile_base[v] + (ys // th) * o.tiles_xy[v][0] + xs // tw).reshape(-1))
    return np.concatenate(out).astype(np.int64) if out else np.zeros(0, np.int64)


def last_composited(vals, ranges, tiles, nc):
    """Record at list position nc - 1 of each pixel's tile, -1 where nc = 0."""
    nc = np.asarray(nc).astype(np.int64)
    start = ranges.reshape(-1, 2)[tiles, 0].astype(np.int64)
    idx = np.maximum(start + nc - 1, 0)
    return np.where(nc > 0, vals[np.minimum(idx, max(vals.size - 1, 0))].astype(np.int64) if vals.size else -1, -1)


def compare_pixel_lists(nc_g, g, o: oracle.Oracle, ref_nc, tiles):
    """Contributor counts are positions in different lists: the records they
    point at must be the same."""
    gr = g["ranges"].reshape(-1, 2)
    glen = (gr[tiles, 1].astype(np.int64) - gr[tiles, 0])
    nc_g = np.asarray(nc_g).astype(np.int64)
    assert np.all(nc_g <= glen), "contributor count beyond the tile's list"
    _, ovals, oranges = o.lists()
    a = last_composited(g["vals"], gr, tiles, nc_g)
    b = last_composited(ovals, oranges, tiles, ref_nc)
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, f"{bad.size} pixels' last composited record differs, first at {bad[:5]}"


def compare_pixels(g, o: oracle.Oracle, ref):
    tiles = pixel_tiles(o)
    compare_pixel_lists(g["ncontrib"], g, o, flat_views(ref["ncontrib"]), tiles)
    tf = flat_views(ref["tfinal"])
    assert np.abs(g["tfinal"] - tf).max() <= IMG_TOL


def examined_counts(g, tiles, stoprec):
    """Entries the GPU forward examines per pixel: up to and including the
    stop entry (which must be in its list), else its whole list."""
    gr = g["ranges"].reshape(-1, 2)
    glen = gr[tiles, 1].astype(np.int64) - gr[tiles, 0]
    stopped = stoprec != 0xFFFFFFFF
    out = glen.copy()
    if stopped.any():
        gp = _pairs(g["keys"], g["vals"])
        order = np.argsort(gp, kind="stable")
        want = (tiles[stopped].astype(np.uint64) << np.uint64(32)) | stoprec[stopped].astype(np.uint64)
        p = np.searchsorted(gp[order], want)
        assert np.all(p < gp.size) and np.array_equal(gp[order][p], want), "a stop entry was dropped"
        out[stopped] = order[p] - gr[tiles[stopped], 0] + 1
    return out


def compare_counters(g, o: oracle.Oracle, ref, with_bwd: bool):
    """The throughput counters: composited pairs equal the oracle's count;
    examined pairs and the contributor sum are those of the GPU's lists."""
    info = g["info"]
    tiles = pixel_tiles(o)
    assert info["blended_pairs"] == int(flat_views(ref["nblend"]).astype(np.int64).sum())
    ex = examined_counts(g, tiles, flat_views(ref["stoprec"]).astype(np.uint32))
    assert info["fwd_pairs"] == int(ex.sum())
    if with_bwd:
        assert info["bwd_pairs"] == int(g["ncontrib"].astype(np.int64).sum())


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


LOG2E = 1.4426950408889634
# GPU record-gradient columns -> (oracle column, factor): the GPU differentiates
# the scaled conic (qa, qb, qc) = -log2(e) (c0/2, c1, c2/2) the blend reads
REC_GRAD_MAP = {"du": (0, 0, 1.0), "dv": (1, 1, 1.0), "dc0": (2, 2, -0.5 * LOG2E), "dc1": (3, 3, -LOG2E),
                "dc2": (4, 4, -0.5 * LOG2E), "dsigma": (5, 5, 1.0), "dz": (6, 9, 1.0), "dr": (8, 6, 1.0),
                "dg": (9, 7, 1.0), "db": (10, 8, 1.0)}
# per-record bar: |gpu - oracle| <= REC_ABS * RMS(field) + REC_REL * |oracle|.
# A record's blend gradient is a binary32 sum over up to a few thousand
# pixels whose terms can cancel; measured on the full-size rig and window
# batches the largest error is 0.3 of this bound, while a wrong term or a
# dropped pixel moves a record by O(1) of its own value.
REC_ABS, REC_REL = 1e-3, 1e-3


def compare_record_grads(g, go, tol=GRAD_TOL):
    """The backward blend's own output: per-record 2D gradients (dL/du, dv,
    conic, opacity, depth, colour) against the oracle's, field by field
    (relative L2 <= tol) and record by record (bounded by the field's RMS)."""
    a = np.asarray(g["grec"], np.float64)
    b = np.asarray(go["grec"], np.float64)
    assert a.shape[0] == b.shape[0], (a.shape, b.shape)
    stats = {}
    for name, (cg, co, fac) in REC_GRAD_MAP.items():
        x, y = a[:, cg] * fac, b[:, co]
        e = rel_l2(x, y)
        rms = float(np.sqrt(np.mean(y * y))) if y.size else 0.0
        worst = float(np.max(np.abs(x - y) / (REC_ABS * rms + REC_REL * np.abs(y) + 1e-30))) if y.size else 0.0
        stats[name] = (e, worst)
        assert e <= tol, f"record grad {name}: rel L2 {e:.3e} > {tol}"
        assert worst <= 1.0, f"record grad {name}: a record is {worst:.2f}x over its bound"
    return stats


def grad_row_quantile(a, b, q=99.9, floor_frac=0.1):
    """q-th percentile over Gaussians of the relative error of the gradient
    row ||a_i - b_i|| / ||b_i||, for rows whose oracle norm exceeds
    floor_frac times the RMS row norm."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    if b.size == 0:
        return 0.0
    a, b = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    nb = np.linalg.norm(b, axis=1)
    floor = floor_frac * float(np.sqrt(np.mean(nb * nb)))
    sel = nb > floor
    if floor == 0:
        return 0.0
    if not sel.any():
        return 0.0
    return float(np.percentile(np.linalg.norm(a[sel] - b[sel], axis=1) / nb[sel], q))


# Per-Gaussian rows.  The preprocess adjoint runs in binary32 (binary64 only
# for large angular footprints).  Its error on a row follows the condition of
# the record's 2D covariance (the conic -> covariance step, dS = -C dC C,
# cancels for elongated footprints) and the cancellation between the
# contributions of pixels inside and outside the rendered region, not the
# row's norm: at full size single rows reach 1.1e-3 RMS absolute, varying run
# to run with the order of the atomics, while the whole tensors stay within
# 1e-4 relative L2.  So two statistics, both failed by an error spread over
# many rows: the 99.9th percentile of the relative error over rows above a
# tenth of the RMS row norm (measured <= 1.3e-3), and the number of rows
# outside ROW_REL |row| + ROW_ABS RMS, at most ROW_OUT_MAX or ROW_OUT_FRAC of
# the touched rows.  An all-zero oracle tensor (rotation-invariant scenes) is
# left to the whole-tensor check.
ROW_Q_TOL = 5e-3
ROW_REL, ROW_ABS = 1e-3, 2e-4
ROW_OUT_MAX, ROW_OUT_FRAC = 5, 2e-3


def compare_grad_rows(g, go, tol=ROW_Q_TOL):
    out = {}
    for name in PARAM_NAMES:
        a, b = np.asarray(g["grads"][name], np.float64), np.asarray(go[name], np.float64)
        e = grad_row_quantile(a, b)
        out[name] = e
        assert e <= tol, f"grad {name}: 99.9th percentile row error {e:.3e} > {tol}"
        if b.size:
            a2, b2 = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
            nb = np.linalg.norm(b2, axis=1)
            rms = float(np.sqrt(np.mean(nb * nb)))
            if rms > 0:
                ratio = np.linalg.norm(a2 - b2, axis=1) / (ROW_REL * nb + ROW_ABS * rms)
                touched = int(np.count_nonzero(nb))
                n_out = int(np.count_nonzero(ratio > 1.0))
                limit = max(ROW_OUT_MAX, int(ROW_OUT_FRAC * touched))
                assert n_out <= limit, (f"grad {name}: {n_out} of {touched} rows outside the per-row bound "
                                        f"(worst {float(ratio.max()):.2f}x)")
    return out


def compare_grads(g, go, tol=GRAD_TOL):
    errs = {}
    for name in PARAM_NAMES + ["pose", "focal"]:
        e = rel_l2(g["grads"][name], go[name])
        errs[name] = e
        assert e <= tol, f"grad {name}: rel L2 {e:.3e} > {tol}"
    return errs
