"""Two-round tile lists (gsr_config.list_prefix < 1): a first round over a
depth prefix of the visible records finishes the tiles whose pixels all stop
inside it; the second round lists and renders the others in full.

What must hold, exactly:
  * images, final transmittance, contributor counts and projected records are
    bit for bit those of the one-round forward, and the gradients agree up to
    the order of the backward's atomic additions (both against the oracle at
    the usual bars too);
  * every tile's two-round list is a prefix of its one-round list, the whole
    list for a tile the second round rendered, and holds every entry its
    pixels examine (the stop entries, the last composited records);
  * the throughput counters equal the one-round forward's.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.scenes import pinhole, look_from  # noqa: E402
from paper_2512_08498_gb300.rasterizer import Rasterizer  # noqa: E402

import _parity as P  # noqa: E402


def _dense_scene(seed=11, n=3000, tile=(16, 16), degree=1):
    """Opaque enough that most tiles saturate (every pixel stops), with a few
    tiles of the second view that never do, and a view over a subset."""
    rng = np.random.default_rng(seed)
    views = [pinhole(96, 64, f=70.0),
             pinhole(80, 48, f=60.0, viewmat=look_from([0.1, 0.0, -0.2], yaw_deg=6.0)),
             pinhole(64, 40, f=50.0, viewmat=look_from([-0.1, 0.05, 0.1], yaw_deg=-5.0, roll_deg=10.0),
                     subset=np.sort(rng.choice(n, n // 2, replace=False)).astype(np.uint32))]
    return scenes.random_scene(seed, n, views, degree, log_scale_range=(-2.5, -0.8), tile=tile,
                               bg=(0.1, 0.2, 0.3))


def _raster(sc, prefix, batch=256):
    r = Rasterizer(tile=sc.tile, batch=batch, sh_degree=sc.sh_degree, bg=sc.bg, device=P.device())
    r.set_config(list_prefix=prefix)
    return r


def _check_prefix_lists(two, one):
    """Each tile's two-round list is a prefix of its one-round list."""
    r2, r1 = two["ranges"].reshape(-1, 2).astype(np.int64), one["ranges"].reshape(-1, 2).astype(np.int64)
    short = 0
    for t in range(r1.shape[0]):
        a = slice(r2[t, 0], r2[t, 1])
        n2, n1 = r2[t, 1] - r2[t, 0], r1[t, 1] - r1[t, 0]
        assert n2 <= n1, f"tile {t}: two-round list longer than the full list"
        assert np.array_equal(two["keys"][a], one["keys"][r1[t, 0]:r1[t, 0] + n2]), f"tile {t}: keys"
        assert np.array_equal(two["vals"][a], one["vals"][r1[t, 0]:r1[t, 0] + n2]), f"tile {t}: records"
        short += int(n2 < n1)
    return short


def _compact(g):
    """The lists the ranges point at, tile after tile in one array (the first
    region also holds stale prefix entries of the tiles left open)."""
    r = g["ranges"].reshape(-1, 2).astype(np.int64)
    idx = np.concatenate([np.arange(a, b) for a, b in r]) if r.size else np.zeros(0, np.int64)
    ln = r[:, 1] - r[:, 0]
    st = np.concatenate([[0], np.cumsum(ln)[:-1]])
    out = dict(g)
    out["keys"], out["vals"] = g["keys"][idx], g["vals"][idx]
    out["ranges"] = np.where((ln > 0)[:, None], np.stack([st, st + ln], 1), 0).astype(np.uint32)
    return out


def _expected_open(sc, o, ref, prefix):
    """Tiles the first round must leave open: those with a pixel that does
    not stop at a record among the first ceil(f V) of the V visible records
    in depth order (ties by record index), from the oracle alone."""
    m = o.mirror()
    vis = np.nonzero((m["flags"] & 1) == 0)[0]
    order = vis[np.lexsort((vis, m["zbits"][vis]))]
    rank = np.full(m["flags"].size, np.iinfo(np.int64).max, dtype=np.int64)
    rank[order] = np.arange(order.size)
    n = order.size
    p = n if prefix >= 1.0 else min(n, max(1, math.ceil(float(np.float32(prefix)) * n)))
    tw, th = sc.tile
    open_tiles = 0
    for s in ref["stoprec"]:
        s = np.asarray(s).astype(np.int64)
        h, w = s.shape
        for y in range(0, h, th):
            for x in range(0, w, tw):
                b = s[y:y + th, x:x + tw]
                stopped = (b != 0xFFFFFFFF).all()
                open_tiles += int(not (stopped and rank[b].max() < p))
    return open_tiles


def _run_both(sc, prefix, batch=256):
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref)
    one = P.run_gpu(sc, raster=_raster(sc, 1.0, batch), grads=up_g)
    two = P.run_gpu(sc, raster=_raster(sc, prefix, batch), grads=up_g)
    return o, ref, up_o, one, two


@pytest.mark.parametrize("prefix", [0.02, 0.15, 0.5, 0.97])
def test_two_rounds_equal_one_round(prefix):
    sc = _dense_scene()
    o, ref, up_o, one, two = _run_both(sc, prefix)
    i1, i2 = one["info"], two["info"]
    assert i1["list_prefix"] == 1.0 and i1["open_tiles"] == 0 and i1["n_instances_second"] == 0
    assert abs(i2["list_prefix"] - prefix) < 1e-7
    for k in ("rgb", "depth", "alpha", "rec", "tfinal", "ncontrib"):
        assert np.array_equal(one[k], two[k]), k
    for k in ("blended_pairs", "fwd_pairs", "bwd_pairs", "warp_entries_bwd", "n_instances_full", "grad_rows",
              "n_visible"):
        assert i1[k] == i2[k], k
    # a warp's walk may end a few entries earlier where its tile's prefix
    # list ends (the all-stopped vote is taken every fourth entry)
    assert i2["warp_entries_fwd"] <= i1["warp_entries_fwd"]
    assert np.linalg.norm(one["grec"] - two["grec"]) <= 1e-6 * np.linalg.norm(one["grec"])
    for k in one["grads"]:
        assert np.linalg.norm(one["grads"][k] - two["grads"][k]) <= 1e-6 * np.linalg.norm(one["grads"][k]), k
    # the lists: prefixes of the full ones, every examined entry kept
    short = _check_prefix_lists(two, one)
    n_tiles = i2["n_tiles"]
    assert 0 <= i2["open_tiles"] <= n_tiles
    # the first region also holds the open tiles' prefix entries, which no
    # range points at any more
    listed = int(np.sum(two["ranges"][:, 1].astype(np.int64) - two["ranges"][:, 0]))
    assert listed <= i2["n_instances"]
    assert i2["list_span"] == two["keys"].size
    assert i2["open_tiles"] == _expected_open(sc, o, ref, prefix)
    if prefix >= 0.15:
        assert short > 0, "no tile ended early"
    assert i2["n_instances_second"] > 0
    tiles = P.pixel_tiles(o)
    c = _compact(two)
    P.compare_lists(c, o, check_reach=False)
    P.compare_pixel_lists(c["ncontrib"], c, o, P.flat_views(ref["ncontrib"]), tiles)
    ex = P.examined_counts(c, tiles, P.flat_views(ref["stoprec"]).astype(np.uint32))
    assert int(ex.sum()) == i1["fwd_pairs"]
    # and against the oracle at the usual bars
    P.compare_images(two, ref)
    go = o.backward(up_o[0], up_o[1], up_o[2], want_grec=True)
    P.compare_grads(two, go)
    P.compare_record_grads(two, go)


@pytest.mark.parametrize("tile,batch", [((32, 8), 128), ((8, 32), 512)])
def test_two_rounds_other_tiles_and_batches(tile, batch):
    sc = _dense_scene(seed=12, n=2500, tile=tile, degree=2)
    o, ref, up_o, one, two = _run_both(sc, 0.2, batch=batch)
    assert two["info"]["open_tiles"] == _expected_open(sc, o, ref, 0.2)
    for k in ("rgb", "depth", "alpha", "tfinal", "ncontrib"):
        assert np.array_equal(one[k], two[k]), k
    for k in one["grads"]:
        assert np.linalg.norm(one["grads"][k] - two["grads"][k]) <= 1e-6 * np.linalg.norm(one["grads"][k]), k
    _check_prefix_lists(two, one)
    P.compare_images(two, ref)


def test_prefix_of_every_record_is_one_round():
    # a fraction whose prefix holds every record makes the first round final
    # everywhere: no open tile, an idle second round
    sc = _dense_scene(seed=13, n=800)
    o, ref, up_o, one, two = _run_both(sc, 0.99999994)
    i2 = two["info"]
    assert i2["open_tiles"] == 0 and i2["n_instances_second"] == 0
    assert i2["n_instances"] == one["info"]["n_instances"]
    c = _compact(two)
    for k in ("rgb", "depth", "alpha", "tfinal", "ncontrib"):
        assert np.array_equal(one[k], two[k]), k
    for k in ("keys", "vals", "ranges"):
        assert np.array_equal(one[k], c[k]), k


def test_sparse_scene_every_tile_open():
    # nothing saturates: every tile goes to the second round, whose lists are
    # the full ones
    sc = scenes.random_scene(14, 300, [pinhole(70, 45, f=60.0), pinhole(33, 31, f=40.0)], 0)
    o, ref, up_o, one, two = _run_both(sc, 0.3)
    i2 = two["info"]
    assert i2["open_tiles"] == i2["n_tiles"]
    r1, r2 = one["ranges"].reshape(-1, 2), two["ranges"].reshape(-1, 2).astype(np.int64)
    for t in range(r1.shape[0]):
        assert np.array_equal(one["keys"][r1[t, 0]:r1[t, 1]], two["keys"][r2[t, 0]:r2[t, 1]])
    for k in ("rgb", "depth", "alpha", "tfinal", "ncontrib"):
        assert np.array_equal(one[k], two[k]), k


def test_empty_scene_two_rounds():
    sc = scenes.random_scene(15, 50, [pinhole(40, 24, f=30.0)], 0, z_range=(-6.0, -1.0))
    o = oracle.Oracle(sc)
    ref = o.forward()
    g = P.run_gpu(sc, raster=_raster(sc, 0.1))
    assert g["info"]["n_visible"] == 0 and g["info"]["n_instances"] == 0
    P.compare_images(g, ref)


def test_automatic_prefix():
    # list_prefix 0: the first forward runs one round and measures; the next
    # ones use the fraction chosen from its saturation histogram
    # large Gaussians (about 24 tiles per record) that saturate early: two
    # rounds pay off and are chosen
    sc = scenes.random_scene(16, 3000, [pinhole(128, 96, f=102.4)], 1, log_scale_range=(-1.8, -0.5),
                             bg=(0.1, 0.2, 0.3))
    r = _raster(sc, 0.0)
    params = P.params_of(sc)
    from paper_2512_08498_gb300.rasterizer import to_camera_views
    cams = to_camera_views(sc.views, P.device())
    rgb0, _, _, s0 = r.forward(params, cams)
    assert s0.info()["list_prefix"] == 1.0
    rgb1, _, _, s1 = r.forward(params, cams)
    f = s1.info()["list_prefix"]
    assert f < 1.0, "a scene whose tiles saturate early should take two rounds"
    rgb2, _, _, s2 = r.forward(params, cams, saved=s1)
    assert torch.equal(rgb1, rgb2)
    assert 0.0 < f <= 1.0
    assert torch.equal(rgb0, rgb1)
    one = P.run_gpu(sc, raster=_raster(sc, 1.0))
    assert np.array_equal(rgb1.cpu().numpy(), one["rgb"])


def test_two_rounds_capacity_growth():
    # lists grown by the synchronous retry in both rounds
    sc = _dense_scene(seed=17, n=2000)
    r = _raster(sc, 0.1)
    from paper_2512_08498_gb300.rasterizer import to_camera_views
    params = P.params_of(sc)
    cams = to_camera_views(sc.views, P.device())
    saved = r.new_saved()
    r.lib.gsr_reserve(r.ctx, saved.h, 1, 1)
    rgb, depth, alpha, saved = r.forward(params, cams, saved=saved)
    assert saved.info()["list_prefix"] < 1.0
    one = P.run_gpu(sc, raster=_raster(sc, 1.0))
    assert np.array_equal(rgb.cpu().numpy(), one["rgb"])


def test_two_rounds_in_a_cuda_graph():
    # both rounds enqueue no host synchronisation: forward and backward are
    # captured once and replayed, with the same images and gradients as the
    # eager calls
    sc = _dense_scene(seed=18, n=2500)
    from paper_2512_08498_gb300.rasterizer import to_camera_views
    r = _raster(sc, 0.3)
    params = P.params_of(sc)
    cams = to_camera_views(sc.views, P.device())
    rgb, depth, alpha, saved = r.forward(params, cams)
    assert 0 < saved.info()["open_tiles"] < saved.info()["n_tiles"]
    ref_rgb = rgb.clone()
    d_rgb = torch.randn_like(rgb) * 1e-3
    grads = r.backward(params, cams, saved, d_rgb)
    ref_g = [g.clone() for g in grads]
    r.set_config(no_sync=True)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            r.forward(params, cams, saved=saved, out=(rgb, depth, alpha))
            r.backward(params, cams, saved, d_rgb, grads=grads)
    for _ in range(3):
        rgb.zero_()
        graph.replay()
    torch.cuda.synchronize()
    r.check(saved)
    assert torch.equal(rgb, ref_rgb)
    for a, b in zip(grads, ref_g):
        assert P.rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5


def test_two_rounds_through_the_autograd_function():
    # the torch.autograd.Function path (pose and focal inputs) under two
    # rounds: gradients against the oracle's and the one-round path's
    from paper_2512_08498_gb300.rasterizer import rasterize, to_camera_views
    sc = _dense_scene(seed=19, n=2000)
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref)
    go = o.backward(*up_o)
    out = {}
    for prefix in (1.0, 0.2):
        r = _raster(sc, prefix)
        params = [p.clone().requires_grad_(True) for p in P.params_of(sc)]
        pose = torch.zeros(len(sc.views), 6, device=P.device(), requires_grad=True)
        focal = torch.zeros(len(sc.views), 2, device=P.device(), requires_grad=True)
        rgb, depth, alpha = rasterize(*params, to_camera_views(sc.views, P.device()), r, pose_delta=pose,
                                      focal_delta=focal)
        d = [torch.from_numpy(x).to(P.device()) for x in up_g]
        loss = (rgb * d[0]).sum() + (depth * d[1]).sum() + (alpha * d[2]).sum()
        loss.backward()
        for name, p in zip(P.PARAM_NAMES, params):
            assert P.rel_l2(p.grad.cpu().numpy(), go[name]) <= P.GRAD_TOL, name
        assert P.rel_l2(pose.grad.cpu().numpy(), go["pose"]) <= P.GRAD_TOL
        assert P.rel_l2(focal.grad.cpu().numpy(), go["focal"]) <= P.GRAD_TOL
        out[prefix] = (rgb.detach().cpu().numpy(), [p.grad.cpu().numpy() for p in params],
                       pose.grad.cpu().numpy())
    assert np.array_equal(out[1.0][0], out[0.2][0])
    for a, b in zip(out[1.0][1], out[0.2][1]):
        assert P.rel_l2(b, a) <= 1e-6
    assert P.rel_l2(out[0.2][2], out[1.0][2]) <= 1e-6
