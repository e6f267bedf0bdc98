"""Pins of the merging oracle (Sec. 3.2, Eq. 7-8): hand-built groups whose
outcome follows from the rule (smallest image-space scale kept, mean colour,
mean depth), the depth gate, reprojection and unprojection in closed form,
the agreement of Eq. 6 and Eq. 8 under the reading, and invariants of the
grouping on random scenes."""
import math

import numpy as np
import pytest

import oracle
from oracle.merging import INSERT, MERGED, REPLACES, UNTOUCHED, REMOVED, KEPT, SH_C0
from paper_2512_08498_gb300.scenes import pinhole, look_from


def _unproject(view, px, py, z):
    """World point seen at pixel centre (px + 1/2, py + 1/2) at camera depth z."""
    V = np.asarray(view.viewmat, np.float64)
    cam = np.array([(px + 0.5 - view.cx) / view.fx * z, (py + 0.5 - view.cy) / view.fy * z, z])
    return V[:3, :3].T @ (cam - V[:3, 3])


def _maps(view, samples, S, d, rng=None):
    H, W = view.height, view.width
    Smap = np.zeros((H, W), np.float32)
    Dmap = np.full((H, W), 5.0, np.float32)
    for (px, py), s, dd in zip(samples, S, d):
        Smap[py, px] = s
        Dmap[py, px] = dd
    gt = (rng.random((3, H, W)) if rng is not None else np.full((3, H, W), 0.5)).astype(np.float32)
    pix = np.array(sorted(py * W + px for px, py in samples), np.int64)
    return pix, Smap, Dmap, gt


def _own_dc(gt, W, px, py):
    return (gt[:, py, px].astype(np.float64) - 0.5) / SH_C0


@pytest.mark.parametrize("finer_existing", [False, True])
def test_pair_keeps_the_finer_primitive(finer_existing):
    rng = np.random.default_rng(1)
    view = pinhole(40, 30, f=35.0, viewmat=look_from([0.1, -0.2, 0.0], yaw_deg=7.0))
    px, py, d, S = 11, 17, 4.0, 0.02                        # sample: s_i = S f / d = 0.175 px
    pix, Smap, Dmap, gt = _maps(view, [(px, py)], [S], [d], rng)
    z_g = 4.1
    s_target = 0.1 if finer_existing else 0.3               # image-space scale of the existing one
    ls = math.log(s_target * z_g / 35.0)
    mu = _unproject(view, px, py, z_g)[None]
    dc = np.array([[0.3, -0.2, 0.9]])
    o = oracle.merging.merge(view, mu, [[ls, ls - 1.0, ls - 2.0]], dc, pix, Smap, Dmap, gt, tau_d=0.5)
    own = _own_dc(gt, 40, px, py)
    mean_dc = (own + dc[0]) / 2
    assert o["pair"][0] == 0
    if finer_existing:
        assert o["sample_action"][0] == MERGED and o["existing_action"][0] == KEPT
        assert np.allclose(o["existing_dc"][0], mean_dc, rtol=0, atol=1e-12)
        assert o["sample_depth"][0] == pytest.approx(d)
    else:
        assert o["sample_action"][0] == REPLACES and o["existing_action"][0] == REMOVED
        assert np.allclose(o["sample_dc"][0], mean_dc, rtol=0, atol=1e-12)
        assert o["sample_depth"][0] == pytest.approx((d + z_g) / 2, rel=1e-6)
        assert o["sample_scale"][0] == pytest.approx(np.float32(S) * (d + z_g) / 2 / d, rel=1e-6)
        assert np.array_equal(o["existing_dc"], dc)


def test_depth_gate_and_unpaired_gaussians():
    view = pinhole(40, 30, f=35.0)
    pix, Smap, Dmap, gt = _maps(view, [(5, 6), (20, 20)], [0.01, 0.01], [3.0, 3.0])
    mus = [_unproject(view, 5, 6, 3.6),       # 0.6 m behind the sample: not the same surface
           _unproject(view, 5, 6, 3.4),       # within 0.5 m: paired
           _unproject(view, 7, 6, 3.0),       # a pixel without a sample
           [0.0, 0.0, -2.0],                  # behind the camera
           _unproject(view, -3, 6, 3.0)]      # left of the image
    ls = np.full((5, 3), math.log(0.001), np.float32)
    o = oracle.merging.merge(view, np.array(mus), ls, np.zeros((5, 3)), pix, Smap, Dmap, gt, tau_d=0.5)
    assert o["pair"].tolist() == [-1, 0, -1, -1, -1]
    assert o["existing_action"].tolist() == [UNTOUCHED, KEPT, UNTOUCHED, UNTOUCHED, UNTOUCHED]
    assert o["sample_action"].tolist() == [MERGED, INSERT]


def test_group_of_several_with_a_tie():
    view = pinhole(32, 24, f=30.0)
    pix, Smap, Dmap, gt = _maps(view, [(9, 9)], [0.05], [2.0])      # s_i = 0.75 px
    z = [2.1, 1.9, 2.05, 2.0]
    s_img = [0.5, 0.4, 0.4, 0.9]                                     # two finest tie: index 1 wins
    mus = np.array([_unproject(view, 9, 9, zz) for zz in z])
    ls = np.array([[math.log(s * zz / 30.0)] * 3 for s, zz in zip(s_img, z)], np.float32)
    ls[2] = ls[1]                                                    # the same scale bits
    mus[2] = mus[1] + np.array([0.0, 0.0, 0.0])                      # and the same depth
    dc = np.arange(12, dtype=np.float64).reshape(4, 3) / 10
    o = oracle.merging.merge(view, mus, ls, dc, pix, Smap, Dmap, gt, tau_d=0.5)
    assert o["existing_action"].tolist() == [REMOVED, KEPT, REMOVED, REMOVED]
    assert o["sample_action"][0] == MERGED
    own = _own_dc(gt, 32, 9, 9)
    assert np.allclose(o["existing_dc"][1], (own + dc.sum(0)) / 5, atol=1e-12)


def test_sample_scale_of_eq6_is_eq8():
    # S = d / (2 sqrt(P) f) (Eq. 6) gives s_i = S f / d = 1 / (2 sqrt(P)) (Eq. 8)
    view = pinhole(16, 16, f=20.0)
    P = 0.37
    d = 3.3
    S = np.float32(d / (2 * math.sqrt(P) * 20.0))
    pix, Smap, Dmap, gt = _maps(view, [(4, 4)], [S], [d])
    s_i = np.float32(np.float32(S * np.float32(20.0)) / np.float32(d))
    assert s_i == pytest.approx(1 / (2 * math.sqrt(P)), rel=1e-6)
    # exactly equal image-space scales (unit scale on the optical axis, f / z = 10 px on both
    # sides): the existing Gaussian is kept
    view = pinhole(16, 16, f=20.0, cx=8.0, cy=8.0)
    pix, Smap, Dmap, gt = _maps(view, [(8, 8)], [1.0], [2.0])
    o = oracle.merging.merge(view, np.array([[0.0, 0.0, 2.0]]), np.zeros((1, 3)), np.zeros((1, 3)), pix, Smap,
                             Dmap, gt)
    assert o["s_existing"][0] == np.float32(10.0)
    assert o["existing_action"][0] == KEPT and o["sample_action"][0] == MERGED


def test_unprojected_samples_reproject_to_their_pixel_centres():
    rng = np.random.default_rng(3)
    view = pinhole(50, 40, f=45.0, cx=23.0, cy=21.5, viewmat=look_from([0.3, 0.1, -0.4], yaw_deg=-12, pitch_deg=5))
    cells = [(int(rng.integers(0, 50)), int(rng.integers(0, 40))) for _ in range(30)]
    cells = sorted(set(cells), key=lambda c: c[1] * 50 + c[0])
    d = rng.uniform(1, 20, len(cells))
    pix, Smap, Dmap, gt = _maps(view, cells, [0.01] * len(cells), d, rng)
    o = oracle.merging.merge(view, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)), pix, Smap, Dmap, gt)
    V = np.asarray(view.viewmat, np.float32).astype(np.float64)
    cam = o["sample_means"] @ V[:3, :3].T + V[:3, 3]
    u = view.fx * cam[:, 0] / cam[:, 2] + view.cx
    v = view.fy * cam[:, 1] / cam[:, 2] + view.cy
    assert np.allclose(u, pix % 50 + 0.5, atol=1e-5) and np.allclose(v, pix // 50 + 0.5, atol=1e-5)
    # (R^T inverts the binary32-rounded rotation up to its 1e-7 departure from orthogonality)
    assert np.allclose(cam[:, 2], Dmap.reshape(-1)[pix], rtol=1e-6, atol=0)
    assert (o["sample_action"] == INSERT).all()


def test_grouping_invariants_on_a_random_scene():
    rng = np.random.default_rng(4)
    view = pinhole(64, 48, f=50.0, viewmat=look_from([0.0, 0.0, -0.5], yaw_deg=4.0))
    W, H = 64, 48
    pix = np.sort(rng.choice(W * H, 600, replace=False))
    Smap = (rng.uniform(0.002, 0.05, (H, W))).astype(np.float32)
    Dmap = rng.uniform(2, 6, (H, W)).astype(np.float32)
    gt = rng.random((3, H, W)).astype(np.float32)
    n = 3000
    sel = rng.choice(W * H, n)
    z = Dmap.reshape(-1)[sel] + rng.normal(0, 0.3, n)
    mus = np.array([_unproject(view, p % W + rng.uniform(-0.45, 0.45), p // W + rng.uniform(-0.45, 0.45), zz)
                    for p, zz in zip(sel, z)])
    ls = rng.uniform(-6, -3, (n, 3)).astype(np.float32)
    dc = rng.normal(0, 0.5, (n, 3))
    o = oracle.merging.merge(view, mus, ls, dc, pix, Smap, Dmap, gt, tau_d=0.4)
    pair = o["pair"]
    assert (pair >= 0).sum() > 100
    for s in range(pix.size):
        members = np.nonzero(pair == s)[0]
        kept = (o["sample_action"][s] == REPLACES) + (o["existing_action"][members] == KEPT).sum()
        if members.size:
            assert kept == 1 and o["sample_action"][s] != INSERT
            assert ((o["existing_action"][members] == REMOVED) | (o["existing_action"][members] == KEPT)).all()
        else:
            assert o["sample_action"][s] == INSERT
    assert (o["existing_action"][pair < 0] == UNTOUCHED).all()
    # relabelling the existing Gaussians relabels the outcome (scales distinct almost surely)
    perm = rng.permutation(n)
    q = oracle.merging.merge(view, mus[perm], ls[perm], dc[perm], pix, Smap, Dmap, gt, tau_d=0.4)
    assert np.array_equal(q["existing_action"], o["existing_action"][perm])
    assert np.array_equal(q["sample_action"], o["sample_action"])
    assert np.allclose(q["sample_dc"], o["sample_dc"], atol=1e-12)
