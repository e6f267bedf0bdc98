"""CUDA path vs the CPU oracle, element by element (needs a GB300 and libgsr).

Small scenes span several tiles with ragged edges, several views with
uneven sizes, Gaussian subsets, all three tile shapes and all three blend
batch sizes; the 10k-Gaussian 256x256 workload is compared in full.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.scenes import pinhole, look_from  # noqa: E402

import _parity as P  # noqa: E402


def _multi_view(seed=7, n=600, degree=3, tile=(16, 16)):
    rng = np.random.default_rng(seed)
    views = [pinhole(70, 45, f=60.0),
             pinhole(48, 40, f=50.0, viewmat=look_from([0.1, -0.05, -0.3], yaw_deg=8.0, pitch_deg=-4.0)),
             pinhole(33, 31, f=40.0, viewmat=look_from([-0.2, 0.1, 0.2], yaw_deg=-10.0),
                     subset=np.sort(rng.choice(n, n // 2, replace=False)).astype(np.uint32)),
             pinhole(64, 36, f=44.0, viewmat=look_from([0.0, 0.05, -0.1], roll_deg=20.0),
                     subset=np.sort(rng.choice(n, n // 3, replace=False)).astype(np.uint32))]
    return scenes.random_scene(seed, n, views, degree, tile=tile, bg=(0.1, 0.2, 0.3))


def _full_check(scene, tile=None, batch=256, grads=True, grad_tol=P.GRAD_TOL, batch_bwd=None):
    o = oracle.Oracle(scene, tile=tile)
    ref = o.forward()
    up_o, up_g = P.upstream(scene, o, ref)
    g = P.run_gpu(scene, tile=tile, batch=batch, grads=up_g if grads else None, batch_bwd=batch_bwd)
    P.compare_records(g, o)
    P.compare_lists(g, o)
    P.compare_pixels(g, o, ref)
    P.compare_counters(g, o, ref, with_bwd=grads)
    errs = P.compare_images(g, ref)
    if grads:
        go = o.backward(up_o[0], up_o[1], up_o[2], want_grec=True)
        P.compare_grads(g, go, tol=grad_tol)
        P.compare_record_grads(g, go, tol=grad_tol)
        P.compare_grad_rows(g, go)
    return g, errs


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
@pytest.mark.parametrize("batch", [128, 256, 512])
def test_multi_view_all_configs(tile, batch):
    sc = _multi_view(tile=tile)
    _full_check(sc, tile=tile, batch=batch)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
@pytest.mark.parametrize("batch,batch_bwd", [(128, 256), (128, 512), (512, 0)])
def test_backward_batches(tile, batch, batch_bwd):
    # the backward's own staging batch (0: the forward's), every tile shape
    _full_check(_multi_view(tile=tile), tile=tile, batch=batch, batch_bwd=batch_bwd)


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_sh_degrees(degree):
    sc = _multi_view(seed=20 + degree, n=300, degree=degree)
    _full_check(sc)


def test_small_box_10k_256():
    sc = scenes.small_box()
    g, errs = _full_check(sc)
    info = g["info"]
    o = oracle.Oracle(sc)
    assert info["n_instances_full"] == int(o.mirror()["tiles"].astype(np.int64).sum()) == o.lists()[0].size
    assert info["n_instances"] == g["keys"].size < info["n_instances_full"]


def test_single_gaussian_closed_form_on_gpu():
    # isotropic Gaussian centred on a pixel corner: the closed-form profile, symmetric
    sc = scenes.Scene("one", np.array([[0, 0, 4.0]], np.float32), np.full((1, 3), math.log(0.5), np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([0.4], np.float32),
                      np.array([[[0.7, 0.2, -0.3]]], np.float32), 0, [pinhole(64, 64, f=64.0)])
    g, _ = _full_check(sc)
    img = g["rgb"][:64 * 64].reshape(64, 64)
    assert np.array_equal(img, img[:, ::-1]) and np.array_equal(img, img[::-1, :])


def test_empty_and_culled_scenes():
    # all Gaussians behind the near plane: background everywhere, no instances
    sc = scenes.Scene("culled", np.array([[0, 0, 0.1], [0, 0, -2.0]], np.float32),
                      np.full((2, 3), -1.0, np.float32), np.array([[1, 0, 0, 0]] * 2, np.float32),
                      np.zeros(2, np.float32), np.zeros((2, 1, 3), np.float32), 0,
                      [pinhole(40, 30, f=40.0)], bg=(0.2, 0.4, 0.6))
    g, _ = _full_check(sc)
    assert g["info"]["n_instances"] == 0 and g["info"]["n_visible"] == 0
    assert np.allclose(g["rgb"].reshape(3, -1), np.array([[0.2], [0.4], [0.6]], np.float32))
    # zero Gaussians
    sc0 = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                       np.zeros((0, 4), np.float32), np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0,
                       [pinhole(17, 9, f=20.0), pinhole(5, 40, f=20.0)], bg=(0.5, 0.5, 0.5))
    g0, _ = _full_check(sc0)
    assert np.all(g0["rgb"] == 0.5)


def test_precull_boundary_off_screen_footprints():
    """Means projected up to three image widths outside the view, some just
    past the near plane or behind the camera, scales up to e^0.5: whether a
    footprint reaches the image decides visibility -- the boundary the
    preprocess pre-cull must never cross.  Records, lists, pixels and
    gradients against the oracle as everywhere else."""
    views = [pinhole(96, 64, f=70.0),
             pinhole(80, 72, f=55.0, cx=20.0, cy=50.0,
                     viewmat=look_from([0.2, -0.1, 0.0], yaw_deg=25.0, roll_deg=10.0))]
    sc = scenes.random_scene(11, 2500, views, 3, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(11)
    n = sc.n
    z = rng.uniform(0.15, 8.0, n)
    z[:100] = rng.uniform(-2.0, 0.2, 100)
    u = rng.uniform(-3 * 96, 4 * 96, n)
    v = rng.uniform(-3 * 64, 4 * 64, n)
    sc.means = np.stack([(u - 48) * np.abs(z) / 70.0, (v - 32) * np.abs(z) / 70.0, z], 1).astype(np.float32)
    sc.log_scales = rng.uniform(-4.0, 0.5, (n, 3)).astype(np.float32)
    g, _ = _full_check(sc)
    info = g["info"]
    assert 0 < info["n_visible"] < info["n_records"] // 2


def test_degenerate_quaternion_and_tiny_views():
    sc = _multi_view(seed=31, n=200)
    sc.quats[5] = 0.0                       # zero quaternion: culled on both sides
    sc.views.append(pinhole(1, 1, f=2.0))   # a 1x1 view
    sc.views.append(pinhole(17, 3, f=9.0, subset=np.zeros(0, np.uint32)))  # empty subset
    o = oracle.Oracle(sc)
    assert o.mirror()["flags"][5] & 1
    _full_check(sc)


def test_depth_ties_and_duplicates():
    # identical Gaussians in two views: ties broken by Gaussian index on both sides
    means = np.array([[0, 0, 3.0]] * 4 + [[0.1, 0.05, 3.0]] * 3, np.float32)
    n = means.shape[0]
    sh = np.random.default_rng(5).uniform(-0.5, 1.0, (n, 1, 3)).astype(np.float32)
    sc = scenes.Scene("ties", means, np.full((n, 3), math.log(0.3), np.float32),
                      np.array([[1, 0, 0, 0]] * n, np.float32), np.zeros(n, np.float32), sh, 0,
                      [pinhole(48, 48, f=48.0), pinhole(48, 48, f=48.0, subset=np.array([1, 2, 5], np.uint32))])
    _full_check(sc)


def _threshold_scene():
    """Gaussians whose alpha sits within a few ulp of the blend's decision
    thresholds: family A at the pixel right of the centre pixel (alpha ~
    1/255; ten scales, twenty Gaussians each), family B at the centre pixel
    with the mean just off the pixel centre (alpha ~ the 0.99 clamp), and a
    large Gaussian behind all of them, so every transmittance matters.  The
    opacities come from the oracle's binary32 projection of the same means
    and scales: sigma* = threshold / 2^P2 at that pixel, then the binary32
    opacity logit of sigma* moved by -10 .. +9 ulp across a family, which
    steps sigma by a few ulp across the threshold."""
    W = H = 96
    f, z = 96.0, 4.0
    view = pinhole(W, H, f=f)
    slots = [(x, y) for y in range(3, H - 3, 5) for x in range(3, W - 3, 5)]
    means, logs, target = [], [], []
    k = 0
    for s_px in np.linspace(0.45, 0.9, 10):
        for _ in range(20):
            px, py = slots[k]
            k += 1
            means.append([(px + 0.5 - W / 2) * z / f, (py + 0.5 - H / 2) * z / f, z])
            logs.append(math.log(s_px * z / f))
            target.append((px + 1, py, 1.0 / 255.0))
    for _ in range(40):
        px, py = slots[k]
        k += 1
        means.append([(px + 0.55 - W / 2) * z / f, (py + 0.54 - H / 2) * z / f, z])
        logs.append(math.log(0.6 * z / f))
        target.append((px, py, 0.99))
    n = len(means)
    means = np.array(means, np.float32)
    logs = np.repeat(np.array(logs, np.float32)[:, None], 3, axis=1)
    quats = np.array([[1, 0, 0, 0]] * n, np.float32)
    sh = np.random.default_rng(12).uniform(-0.5, 1.0, (n, 1, 3)).astype(np.float32)
    probe = scenes.Scene("thresholds_probe", means, logs, quats, np.zeros(n, np.float32), sh, 0, [view])
    rec = oracle.Oracle(probe).mirror()["blend"]          # u, v, qa, qb, qc, sigma (binary32)
    opac = np.empty(n, np.float32)
    f32 = np.float32
    for i, (px, py, thr) in enumerate(target):
        u, v, qa, qb, qc = (f32(x) for x in rec[i, :5])
        dx, dy = f32(f32(px) + f32(0.5)) - u, f32(f32(py) + f32(0.5)) - v
        p2 = f32(dx * f32(f32(qa * dx) + f32(qb * dy))) + f32(f32(qc * dy) * dy)
        sig = thr / oracle.exp2_f32(float(min(p2, f32(0.0))))
        o = f32(math.log(sig / (1.0 - sig)))
        for _ in range(abs(i % 20 - 10)):
            o = np.nextafter(o, f32(np.inf) if i % 20 >= 10 else f32(-np.inf))
        opac[i] = o
    means = np.vstack([means, [[0.0, 0.0, 8.0]]]).astype(np.float32)
    logs = np.vstack([logs, [[math.log(40.0 * 8.0 / f)] * 3]]).astype(np.float32)
    quats = np.vstack([quats, [[1, 0, 0, 0]]]).astype(np.float32)
    opac = np.append(opac, np.float32(0.0))
    sh = np.vstack([sh, [[[0.3, 0.2, 0.1]]]]).astype(np.float32)
    return scenes.Scene("thresholds", means, logs, quats, opac, sh, 0, [view])


def test_backward_decisions_at_alpha_thresholds():
    # The backward takes alpha's value from the hardware 2^x and re-takes the
    # 1/255 and 0.99 decisions with the contract's exponential near them; a
    # flipped decision would drop or add a pair worth several percent of its
    # Gaussian's opacity gradient.
    sc = _threshold_scene()
    g, _ = _full_check(sc)
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, _ = P.upstream(sc, o, ref)
    go = o.backward(up_o[0], up_o[1], up_o[2])
    a, b = g["grads"]["opacity_logits"], go["opacity_logits"]
    scale = np.median(np.abs(b[:-1]))
    assert scale > 0
    bad = np.nonzero(np.abs(a - b) > 1e-3 * (np.abs(b) + scale))[0]
    assert bad.size == 0, f"opacity gradients differ at {bad[:8]}: {a[bad[:4]]} vs {b[bad[:4]]}"


def test_many_views_max():
    views = [pinhole(20 + (i % 7), 18 + (i % 5), f=24.0,
                     viewmat=look_from([0.02 * i, 0.0, -0.05 * (i % 3)], yaw_deg=(i % 9) - 4.0))
             for i in range(64)]
    sc = scenes.random_scene(41, 150, views, 1, bg=(0.0, 0.1, 0.0))
    _full_check(sc)


@pytest.mark.parametrize("degree", [2, 3])
def test_two_groups_of_many_views(degree):
    # groups of >= 12 views take the backward's transposed SH sums: a first
    # group of 14 views (plain row stores) and a second of 13 over a subset
    # (reductions onto the first group's rows), runs of records that cross
    # warps; SH degree 2 (27 outputs per row, a ragged lane split) and 3
    rng = np.random.default_rng(43)
    n = 400
    sub = np.sort(rng.choice(n, 3 * n // 4, replace=False)).astype(np.uint32)
    views = [pinhole(24 + (i % 5), 20 + (i % 3), f=26.0,
                     viewmat=look_from([0.015 * i, 0.01 * (i % 4), -0.04 * (i % 3)], yaw_deg=(i % 7) - 3.0),
                     subset=None if i < 14 else sub)
             for i in range(27)]
    sc = scenes.random_scene(43, n, views, degree, bg=(0.1, 0.0, 0.2))
    _full_check(sc)


def test_batched_equals_per_view():
    sc = _multi_view(seed=50, n=500)
    gb = P.run_gpu(sc)
    offs = [0]
    for v in sc.views:
        offs.append(offs[-1] + v.width * v.height)
    for i, v in enumerate(sc.views):
        one = scenes.Scene(sc.name, sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh, sc.sh_degree,
                           [v], tile=sc.tile, bg=sc.bg)
        g1 = P.run_gpu(one)
        a, b = offs[i], offs[i + 1]
        assert np.array_equal(g1["rgb"], gb["rgb"][3 * a: 3 * b])
        assert np.array_equal(g1["ncontrib"], gb["ncontrib"][a:b])


def test_forward_without_pair_counters():
    # GSR_FLAG_NO_PAIR_COUNTS drops only the two statistics: images, lists,
    # records and pixels are bit for bit those of the counting forward; the
    # gradients agree up to the order of the backward's atomic additions
    from paper_2512_08498_gb300.rasterizer import Rasterizer
    sc = _multi_view(seed=55, n=600)
    o = oracle.Oracle(sc)
    ups = P.upstream(sc, o, o.forward())[1]
    res = []
    for counts in (True, False):
        r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg, device=P.device())
        r.set_config(pair_counts=counts)
        res.append(P.run_gpu(sc, raster=r, grads=ups))
    a, b = res
    for k in ("rgb", "depth", "alpha", "keys", "vals", "ranges", "rec", "tfinal", "ncontrib"):
        assert np.array_equal(a[k], b[k]), k
    assert np.linalg.norm(a["grec"] - b["grec"]) <= 1e-6 * np.linalg.norm(a["grec"])
    for k in a["grads"]:
        assert np.linalg.norm(a["grads"][k] - b["grads"][k]) <= 1e-6 * np.linalg.norm(a["grads"][k]), k
    ia, ib = a["info"], b["info"]
    assert ia["blended_pairs"] > 0 and ia["fwd_pairs"] >= ia["blended_pairs"]
    assert ib["blended_pairs"] == 0 and ib["fwd_pairs"] == 0
    assert ia["warp_entries_fwd"] == ib["warp_entries_fwd"] and ia["bwd_pairs"] == ib["bwd_pairs"]


def test_capacity_growth():
    # start with tiny internal buffers: the forward must grow them and re-run
    sc = _multi_view(seed=60, n=400)
    from paper_2512_08498_gb300.rasterizer import Rasterizer
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    s = r.new_saved()
    r.lib.gsr_reserve(r.ctx, s.h, 1, 1)
    o = oracle.Oracle(sc)
    ref = o.forward()
    params = P.params_of(sc)
    from paper_2512_08498_gb300.rasterizer import to_camera_views
    rgb, _, _, s = r.forward(params, to_camera_views(sc.views), saved=s)
    assert np.abs(rgb.cpu().numpy() - P.flat_views(ref["rgb"])).max() <= P.IMG_TOL


def test_autograd_function_and_pose_input():
    from paper_2512_08498_gb300.rasterizer import Rasterizer, rasterize, to_camera_views
    sc = _multi_view(seed=70, n=300)
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref)
    r = Rasterizer(tile=sc.tile, sh_degree=sc.sh_degree, bg=sc.bg)
    params = [p.clone().requires_grad_(True) for p in P.params_of(sc)]
    pose = torch.zeros(len(sc.views), 6, device=P.device(), requires_grad=True)
    focal = torch.zeros(len(sc.views), 2, device=P.device(), requires_grad=True)
    rgb, depth, alpha = rasterize(*params, to_camera_views(sc.views), r, pose_delta=pose, focal_delta=focal)
    d = [torch.from_numpy(x).to(P.device()) for x in up_g]
    loss = (rgb * d[0]).sum() + (depth * d[1]).sum() + (alpha * d[2]).sum()
    loss.backward()
    go = o.backward(*up_o)
    for name, p in zip(P.PARAM_NAMES, params):
        assert P.rel_l2(p.grad.cpu().numpy(), go[name]) <= P.GRAD_TOL, name
    assert P.rel_l2(pose.grad.cpu().numpy(), go["pose"]) <= P.GRAD_TOL
    assert P.rel_l2(focal.grad.cpu().numpy(), go["focal"]) <= P.GRAD_TOL


def test_autograd_function_depth_only_loss():
    """A loss on the depth image alone: autograd passes no rgb gradient, the
    Function supplies zeros; the gradients equal the oracle's under a zero
    rgb and alpha upstream."""
    from paper_2512_08498_gb300.rasterizer import Rasterizer, rasterize, to_camera_views
    sc = _multi_view(seed=71, n=300)
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref, seed=3)
    r = Rasterizer(tile=sc.tile, sh_degree=sc.sh_degree, bg=sc.bg)
    params = [p.clone().requires_grad_(True) for p in P.params_of(sc)]
    pose = torch.zeros(len(sc.views), 6, device=P.device(), requires_grad=True)
    _, depth, _ = rasterize(*params, to_camera_views(sc.views), r, pose_delta=pose)
    (depth * torch.from_numpy(up_g[1]).to(P.device())).sum().backward()
    zeros = [np.zeros_like(x) for x in up_o[0]]
    go = o.backward(zeros, up_o[1], None)
    for name, p in zip(P.PARAM_NAMES, params):
        assert P.rel_l2(p.grad.cpu().numpy(), go[name]) <= P.GRAD_TOL, name
    assert P.rel_l2(pose.grad.cpu().numpy(), go["pose"]) <= P.GRAD_TOL


def test_autograd_function_rejects_a_nonzero_delta():
    from paper_2512_08498_gb300.rasterizer import Rasterizer, rasterize, to_camera_views
    sc = _multi_view(seed=72, n=50)
    r = Rasterizer(tile=sc.tile, sh_degree=sc.sh_degree, bg=sc.bg)
    params = P.params_of(sc)
    pose = torch.zeros(len(sc.views), 6, device=P.device())
    pose[1, 4] = 1e-3
    with pytest.raises(ValueError):
        rasterize(*params, to_camera_views(sc.views), r, pose_delta=pose)
    with pytest.raises(ValueError):
        rasterize(*params, to_camera_views(sc.views), r, focal_delta=torch.ones(len(sc.views), 2,
                                                                                 device=P.device()))


def test_cuda_graph_capture_replay():
    from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views
    sc = _multi_view(seed=80, n=400)
    r = Rasterizer(tile=sc.tile, sh_degree=sc.sh_degree, bg=sc.bg)
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    rgb, depth, alpha, saved = r.forward(params, cams)           # sizes the buffers
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


@pytest.mark.parametrize("n,offset", [(1, 0), (7, 0), (4099, 0), (3 * 257 * 131, 1), (1 << 20, 0)])
def test_l1_loss_grad_helper(n, offset):
    """The L1 helper against its definition: loss = mean |rgb - target|,
    dl = sign(rgb - target) / n (0 where equal); ragged lengths and a
    misaligned start take the scalar path."""
    import torch
    from paper_2512_08498_gb300.rasterizer import l1_loss_grad
    dev = P.device()
    rng = np.random.default_rng(n)
    a = rng.random(n + offset).astype(np.float32)
    b = rng.random(n + offset).astype(np.float32)
    b[offset::5] = a[offset::5]                          # exact ties give a zero gradient
    ta = torch.from_numpy(a).to(dev)[offset:]
    tb = torch.from_numpy(b).to(dev)[offset:]
    dl = torch.empty(n, device=dev)
    loss = torch.zeros(1, device=dev)
    l1_loss_grad(ta, tb, dl, loss)
    d = a[offset:].astype(np.float64) - b[offset:].astype(np.float64)
    inv = np.float32(1.0) / np.float32(n)
    expect = np.where(d > 0, inv, np.where(d < 0, -inv, np.float32(0))).astype(np.float32)
    assert np.array_equal(dl.cpu().numpy(), expect)
    assert abs(float(loss.item()) - np.abs(d).mean()) <= 1e-5 * max(1.0, np.abs(d).mean())
