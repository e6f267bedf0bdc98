"""GPU parity of the insertion probability and scale initialisation
(Sec. 3.2, Eq. 4-6) against the oracle: the insertion decisions and the
ascending index list bit-exact against the oracle's binary32 mirror, P_a and
the scales within 1e-5 of its double-precision values."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.scenes import pinhole  # noqa: E402

import _parity as P  # noqa: E402

pytestmark = pytest.mark.gpu

PA_TOL = 1e-5
SCALE_RTOL = 1e-5


def _run(views, gt_list, ren_list, depth_list, sigma=1.0, tau_a=0.2, index_cap=None):
    import torch
    from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views
    dev = P.device()
    r = Rasterizer(device=dev)
    cams = to_camera_views(views, dev)
    gt = torch.from_numpy(np.concatenate([g.reshape(-1) for g in gt_list])).to(dev)
    ren = torch.from_numpy(np.concatenate([g.reshape(-1) for g in ren_list])).to(dev)
    dep = torch.from_numpy(np.concatenate([d.reshape(-1) for d in depth_list])).to(dev)
    p_a, scale, index, count = r.insertion(gt, ren, dep, cams, sigma=sigma, tau_a=tau_a, index_cap=index_cap)
    return p_a.cpu().numpy(), scale.cpu().numpy(), index.cpu().numpy().view(np.uint32), count


def _expect(views, gt_list, ren_list, depth_list, sigma=1.0, tau_a=0.2):
    pa, sc, ins = [], [], []
    for v, g, r, d in zip(views, gt_list, ren_list, depth_list):
        o = oracle.insertion(g, r, d, v.fx, sigma=sigma, tau_a=tau_a)
        pa.append(o["p_a"].reshape(-1)); sc.append(o["scale"].reshape(-1)); ins.append(o["inserted"].reshape(-1))
    return np.concatenate(pa), np.concatenate(sc), np.concatenate(ins)


def _compare(got, exp):
    p_a, scale, index, count = got
    pa64, sc64, ins = exp
    assert np.abs(p_a - pa64).max() <= PA_TOL
    idx = np.nonzero(ins)[0].astype(np.uint32)
    assert count == idx.size
    assert np.array_equal(index[: min(count, index.size)], idx[: index.size])
    assert (scale[~ins] == 0).all()
    if idx.size:
        rel = np.abs(scale[ins] - sc64[ins]) / np.abs(sc64[ins])
        assert rel.max() <= SCALE_RTOL
    return idx.size


def _images(rng, views):
    gts, rens, deps = [], [], []
    for v in views:
        h, w = v.height, v.width
        gt = rng.random((3, h, w)).astype(np.float32)
        ren = np.clip(gt + rng.normal(0, 0.08, gt.shape), 0, 1).astype(np.float32)
        ren[:, h // 4: h // 2, w // 4: w // 2] = 0.5    # a flat, poorly reconstructed patch
        gts.append(gt); rens.append(ren)
        deps.append((1.0 + 10.0 * rng.random((h, w))).astype(np.float32))
    return gts, rens, deps


@pytest.mark.parametrize("sigma,tau_a", [(0.5, 0.2), (1.0, 0.2), (2.0, 0.01)])
def test_ragged_views_all_sigmas(sigma, tau_a):
    # (the unnormalised LoG falls like sigma^-4: a wider filter needs a lower threshold)
    rng = np.random.default_rng(int(sigma * 10))
    views = [pinhole(70, 45, f=60.0), pinhole(48, 40, f=50.0), pinhole(33, 31, f=40.0), pinhole(1, 1, f=5.0),
             pinhole(5, 200, f=80.0)]
    g, r, d = _images(rng, views)
    n = _compare(_run(views, g, r, d, sigma=sigma, tau_a=tau_a), _expect(views, g, r, d, sigma=sigma, tau_a=tau_a))
    assert n > 0


def test_index_capacity_and_threshold():
    rng = np.random.default_rng(7)
    views = [pinhole(64, 48, f=60.0), pinhole(40, 40, f=60.0)]
    g, r, d = _images(rng, views)
    exp = _expect(views, g, r, d, tau_a=0.05)
    n = int(exp[2].sum())
    assert n > 100
    got = _run(views, g, r, d, tau_a=0.05, index_cap=n // 3)
    assert got[3] == n and got[2].size == n // 3
    _compare(got, exp)


def test_equal_images_insert_nothing():
    rng = np.random.default_rng(8)
    views = [pinhole(50, 30, f=40.0)]
    g, _, d = _images(rng, views)
    p_a, scale, index, count = _run(views, g, g, d)
    assert count == 0 and (p_a == 0).all() and (scale == 0).all()


def test_on_rendered_rig_views_full_size():
    """The 1M-Gaussian rig: ground truth = the seeded targets, rendering =
    the rasterizer's own output, distance = its normalised depth; every
    pixel of all six 1600x900 views against the oracle."""
    import torch
    from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views
    sc = scenes.rig6()
    dev = P.device()
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg, device=dev)
    params = P.params_of(sc, dev)
    cams = to_camera_views(sc.views, dev)
    rgb, depth, alpha, saved = r.forward(params, cams)
    dist = (depth / alpha.clamp_min(1e-3)).clamp_min(0.2)
    gts = sc.targets()
    offs = np.cumsum([0] + [v.width * v.height for v in sc.views])
    rgb_h, dist_h = rgb.cpu().numpy(), dist.cpu().numpy()
    rens = [rgb_h[3 * offs[i]: 3 * offs[i + 1]].reshape(3, v.height, v.width) for i, v in enumerate(sc.views)]
    deps = [dist_h[offs[i]: offs[i + 1]].reshape(v.height, v.width) for i, v in enumerate(sc.views)]
    gt_t = torch.from_numpy(np.concatenate([t.reshape(-1) for t in gts]).astype(np.float32)).to(dev)
    p_a, scale, index, count = r.insertion(gt_t, rgb, dist, cams)
    got = (p_a.cpu().numpy(), scale.cpu().numpy(), index.cpu().numpy().view(np.uint32), count)
    n = _compare(got, _expect(sc.views, [t.astype(np.float32) for t in gts], rens, deps))
    assert n > 1000
