"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test checks the oracle against mathematics that fixes the answer:
closed forms of single/two-Gaussian renders, library routines (numpy exp,
scipy spherical harmonics), brute-force compositing without tiles, the exact
invariants of the blend (alpha clamp 0.99, 1/255 skip, 1e-4 stop, depth ties
by index), central finite differences of the FP64 forward against the
analytic adjoint, and the agreement of the binary32 decision mirror with a
double-precision evaluation of the same decisions.
"""
import math

import numpy as np
import pytest

from paper_2512_08498_gb300 import scenes
from paper_2512_08498_gb300.scenes import Scene, View, pinhole, look_from

pytestmark = pytest.mark.usefixtures("oracle_lib")

ALPHA_MIN = float(np.float32(1.0 / 255.0))


def _one(means, log_scales, quats=None, opac=None, sh=None, views=None, degree=0, tile=(16, 16), bg=(0, 0, 0)):
    means = np.atleast_2d(np.asarray(means, np.float32))
    n = means.shape[0]
    log_scales = np.broadcast_to(np.asarray(log_scales, np.float32), (n, 3)).copy()
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.atleast_2d(np.asarray(quats, np.float32))
    opac = np.full(n, 3.0, np.float32) if opac is None else np.asarray(opac, np.float32).reshape(n)
    K = (degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(n, K, 3)
    views = views or [pinhole(64, 64, f=64.0)]
    return Scene("t", means, log_scales, quats, opac, sh, degree, views, tile=tile, bg=bg)


def _sigmoid(x):
    return 1.0 / (1.0 + math.exp(-float(np.float32(x))))


def _s(x):
    """exp of a log-scale as stored (binary32)."""
    return math.exp(float(np.float32(math.log(x))))


# ---------------------------------------------------------------------------
# binary32 exponentials vs numpy (library routine), <= 2 ulp
# ---------------------------------------------------------------------------

def _ulp_err(got, x):
    ref = np.exp(np.float64(x))
    ulp = np.spacing(np.float32(ref)).astype(np.float64)
    return abs(np.float64(got) - ref) / ulp


def test_exp_f32_within_2ulp(oracle_lib):
    xs = np.concatenate([np.linspace(-87.0, 88.0, 20001), np.random.default_rng(0).uniform(-20, 20, 5000)])
    worst = max(_ulp_err(oracle_lib.exp_f32(float(np.float32(x))), float(np.float32(x))) for x in xs)
    assert worst <= 2.0, worst
    assert oracle_lib.exp_f32(0.0) == 1.0


def test_exp2_f32_within_2ulp(oracle_lib):
    ys = np.concatenate([np.linspace(-126.0, 0.0, 20001), np.random.default_rng(1).uniform(-10, 3, 5000)])
    worst = 0.0
    for y in ys:
        y32 = float(np.float32(y))
        got = oracle_lib.exp2_f32(y32)
        ref = 2.0 ** y32
        ulp = float(np.spacing(np.float32(ref)))
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 2.0, worst
    # exact powers of two
    for k in range(-126, 1):
        assert oracle_lib.exp2_f32(float(k)) == 2.0 ** k


# ---------------------------------------------------------------------------
# spherical harmonics vs scipy (library routine), sign convention (-1)^m
# ---------------------------------------------------------------------------

def _real_sh_scipy(l, m, d):
    from scipy.special import sph_harm_y
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return float(np.real(sph_harm_y(l, 0, theta, phi)))
    if m > 0:
        return float(math.sqrt(2) * (-1) ** m * np.real(sph_harm_y(l, m, theta, phi)))
    return float(math.sqrt(2) * (-1) ** m * np.imag(sph_harm_y(l, -m, theta, phi)))


def test_sh_basis_matches_scipy(oracle_lib):
    rng = np.random.default_rng(2)
    # the standard real harmonic of band 1, m = 1 is +sqrt(3/4pi) x
    assert abs(_real_sh_scipy(1, 1, (1.0, 0.0, 0.0)) - math.sqrt(3 / (4 * math.pi))) < 1e-12
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        b64, db = oracle_lib.sh_basis_f64(3, d)
        b32 = oracle_lib.sh_basis_f32(3, d.astype(np.float32))
        i = 0
        for l in range(4):
            for m in range(-l, l + 1):
                ref = (-1) ** m * _real_sh_scipy(l, m, d)
                assert abs(b64[i] - ref) < 1e-12, (l, m, b64[i], ref)
                assert abs(b32[i] - ref) < 2e-6, (l, m)
                i += 1
        # Jacobian of the FP64 basis vs central differences
        h = 1e-6
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd = (oracle_lib.sh_basis_f64(3, d + e)[0] - oracle_lib.sh_basis_f64(3, d - e)[0]) / (2 * h)
            assert np.allclose(db[:, j], fd, atol=1e-8)


# ---------------------------------------------------------------------------
# projection closed forms
# ---------------------------------------------------------------------------

def test_isotropic_gaussian_projection_and_radius(oracle_lib):
    f, z, ls = 64.0, 4.0, math.log(0.25)
    sc = _one([0, 0, z], ls, views=[pinhole(64, 64, f=f)])
    o = oracle_lib.Oracle(sc)
    m, r = o.mirror(), o.rec64()
    s = _s(0.25)
    a = (f * s / z) ** 2 + 0.3
    assert np.allclose(r[0, :5], [32.0, 32.0, 1 / a, 0.0, 1 / a], rtol=1e-12, atol=1e-12)
    assert r[0, 9] == pytest.approx(z)
    assert m["radius"][0] == math.ceil(3 * math.sqrt(a + math.sqrt(0.1)))
    assert np.allclose(m["conic"][0], [1 / a, 0, 1 / a], rtol=1e-6, atol=1e-7)
    assert m["zbits"][0] == np.float32(z).view(np.uint32)
    assert r[0, 5] == pytest.approx(_sigmoid(3.0), rel=1e-14)


def test_rotated_camera_projection(oracle_lib):
    # camera at the origin yawed +90 deg about y looks along world +x
    vm = look_from([0, 0, 0], yaw_deg=90.0)
    sc = _one([5.0, 0.5, 0.0], math.log(0.05), views=[pinhole(64, 64, f=64.0, viewmat=vm)])
    r = oracle_lib.Oracle(sc).rec64()
    assert r[0, 0] == pytest.approx(32.0, abs=1e-9)
    assert r[0, 1] == pytest.approx(32.0 + 64.0 * 0.5 / 5.0, abs=1e-9)
    assert r[0, 9] == pytest.approx(5.0, abs=1e-12)


def test_quaternion_convention_wxyz(oracle_lib):
    # 90 deg about camera z swaps the x and y extents of an anisotropic Gaussian
    f, z, sx, sy = 64.0, 4.0, 0.4, 0.1
    q = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    sc = _one([0, 0, z], [math.log(sx), math.log(sy), math.log(0.2)], quats=[q],
              views=[pinhole(64, 64, f=f)])
    r = oracle_lib.Oracle(sc).rec64()
    a = (f * _s(sy) / z) ** 2 + 0.3
    c = (f * _s(sx) / z) ** 2 + 0.3
    assert np.allclose(r[0, 2:5], [1 / a, 0, 1 / c], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("xz,s", [(0.4, 0.2), (1.0, 1.0)])
def test_off_axis_jacobian_and_guard(oracle_lib, xz, s):
    # isotropic Gaussian at x/z = xz: Sigma2D_xx = (f s / z)^2 (1 + t^2) + 0.3 with t = clamp(xz, +-lim)
    f, z = 64.0, 4.0
    sc = _one([xz * z, 0.0, z], math.log(s), views=[pinhole(64, 64, f=f)])
    o = oracle_lib.Oracle(sc)
    r = o.rec64()
    lim = 1.3 * 32.0 / 64.0
    s = _s(s)
    t = max(-lim, min(lim, float(np.float32(xz * z)) / z))
    sxx = (f * s / z) ** 2 * (1 + t * t) + 0.3
    syy = (f * s / z) ** 2 + 0.3
    sxy = 0.0
    det = sxx * syy - sxy * sxy
    assert r[0, 2] == pytest.approx(syy / det, rel=1e-10)
    assert r[0, 4] == pytest.approx(sxx / det, rel=1e-10)
    clamped = bool(o.mirror()["flags"][0] & 4)
    assert clamped == (xz > lim)


# ---------------------------------------------------------------------------
# blend closed forms and invariants
# ---------------------------------------------------------------------------

def test_single_gaussian_profile_closed_form(oracle_lib):
    f, z, s, op = 64.0, 4.0, 0.5, 0.4
    k0 = 0.7
    sh = np.array([[[k0, 0.2, -0.3]]], np.float32)
    bg = (0.1, 0.2, 0.3)
    sc = _one([0, 0, z], math.log(s), opac=[op], sh=sh, bg=bg, views=[pinhole(64, 64, f=f)])
    out = oracle_lib.Oracle(sc).forward()
    a = (f * _s(s) / z) ** 2 + 0.3
    col = 0.5 + np.array([k0, 0.2, -0.3], np.float32).astype(np.float64) / (2 * math.sqrt(math.pi))
    col = np.maximum(col, 0)
    ys, xs = np.mgrid[0:64, 0:64]
    d2 = (xs + 0.5 - 32.0) ** 2 + (ys + 0.5 - 32.0) ** 2
    alpha = np.minimum(0.99, _sigmoid(op) * np.exp(-0.5 * d2 / a))
    rad = math.ceil(3 * math.sqrt(a + math.sqrt(0.1)))
    inside = (np.abs(xs // 16 - 2) <= 4)  # the whole 64x64 view is covered by the rect here
    assert rad * 2 < 64 * 4 and inside.all()
    keep = alpha >= ALPHA_MIN
    alpha = np.where(keep, alpha, 0.0)
    margin = np.abs(np.where(keep, alpha, _sigmoid(op) * np.exp(-0.5 * d2 / a)) - ALPHA_MIN) > 1e-6
    for ch in range(3):
        exp_img = col[ch] * alpha + (1 - alpha) * bg[ch]
        assert np.allclose(out["rgb"][0][ch][margin], exp_img[margin], atol=1e-12)
    assert np.allclose(out["alpha"][0][margin], alpha[margin], atol=1e-12)
    assert np.allclose(out["depth"][0][margin], (z * alpha)[margin], atol=1e-12)
    # the Gaussian is centred on the corner shared by pixels (31,31)..(32,32): mirror symmetry
    img = out["rgb"][0][0]
    assert np.array_equal(img, img[:, ::-1]) and np.array_equal(img, img[::-1, :])
    c4 = [img[31, 31], img[31, 32], img[32, 31], img[32, 32]]
    assert max(c4) - min(c4) == 0.0


def test_two_on_axis_gaussians_composite(oracle_lib):
    # nearer Gaussian listed second: depth order, not index order, decides
    f = 64.0
    means = [[0, 0, 6.0], [0, 0, 3.0]]
    sh = np.array([[[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]]], np.float32)
    bg = (0.05, 0.1, 0.15)
    sc = _one(means, math.log(0.3), opac=[0.5, -0.2], sh=sh, bg=bg, views=[pinhole(64, 64, f=f)])
    out = oracle_lib.Oracle(sc).forward()
    c0 = 1 / (2 * math.sqrt(math.pi))
    px = (31, 31)
    def alpha_of(z, op):
        a = (f * _s(0.3) / z) ** 2 + 0.3
        d2 = 0.5   # pixel centre (31.5, 31.5) vs. mean (32, 32)
        return min(0.99, _sigmoid(op) * math.exp(-0.5 * d2 / a))
    a_near, a_far = alpha_of(3.0, -0.2), alpha_of(6.0, 0.5)
    col_near = np.array([0.5, 0.5 + c0, 0.5])
    col_far = np.array([0.5 + c0, 0.5, 0.5])
    exp_rgb = col_near * a_near + col_far * a_far * (1 - a_near) + np.array(bg) * (1 - a_near) * (1 - a_far)
    got = np.array([out["rgb"][0][ch][px] for ch in range(3)])
    assert np.allclose(got, exp_rgb, atol=1e-12)
    assert out["depth"][0][px] == pytest.approx(3.0 * a_near + 6.0 * a_far * (1 - a_near), abs=1e-12)
    assert out["ncontrib"][0][px] == 2


def test_alpha_clamp_and_early_stop(oracle_lib):
    # huge opacity at the centre: alpha clamps at 0.99 and T stops after 2 entries
    # (T: 1 -> 0.01 -> 1e-4 not below the stop?)  use alpha 0.99 and count stops exactly
    f = 64.0
    zs = [2.0, 3.0, 4.0, 5.0]
    n = len(zs)
    sc = _one([[0, 0, z] for z in zs], math.log(1.0), opac=[12.0] * n,
              sh=np.zeros((n, 1, 3), np.float32), views=[pinhole(64, 64, f=f)])
    o = oracle_lib.Oracle(sc)
    out = o.forward()
    px = (31, 31)
    # binary32 transmittance sequence under the 0.99 clamp
    T = np.float32(1.0)
    k_blended = 0
    for k in range(n):
        Tn = np.float32(T * np.float32(np.float32(1.0) - np.float32(0.99)))
        if Tn < np.float32(1e-4):
            break
        T = Tn
        k_blended = k + 1
    assert out["ncontrib"][0][px] == k_blended
    assert out["alpha"][0][px] == pytest.approx(1 - 0.01 ** k_blended, rel=1e-12)
    assert out["tfinal"][0].min() >= 1e-4 * (1 - 1e-6)


def test_stop_rule_with_alpha_095(oracle_lib):
    f = 64.0
    n = 5
    zs = [2.0 + k for k in range(n)]
    # sigma * G at the centre pixel ~= 0.95 for every Gaussian: choose the logit from the closed form
    logits, alphas = [], []
    for z in zs:
        a = (f * 1.0 / z) ** 2 + 0.3
        G = math.exp(-0.5 * 0.5 / a)
        sig = 0.95 / G
        logits.append(math.log(sig / (1 - sig)))
    sh = np.stack([np.array([[float(k), 0, 0]], np.float32) for k in range(n)])
    sc = _one([[0, 0, z] for z in zs], math.log(1.0), opac=logits, sh=sh, views=[pinhole(64, 64, f=f)])
    out = oracle_lib.Oracle(sc).forward()
    px = (31, 31)
    # T: 1, .05, .0025, 1.25e-4, 6.25e-6 -> the 4th entry is the stop entry, 3 blended
    assert out["ncontrib"][0][px] == 3
    assert out["nexam"][0][px] == 4
    c0 = 1 / (2 * math.sqrt(math.pi))
    cols = [0.5 + k * c0 for k in range(n)]
    a = 0.95
    exp_r = sum(cols[k] * a * (1 - a) ** k for k in range(3))
    assert out["rgb"][0][0][px] == pytest.approx(exp_r, rel=1e-5)


def test_skip_below_1_over_255(oracle_lib):
    # a single faint Gaussian with sigma < 1/255 never contributes
    sc = _one([0, 0, 4.0], math.log(0.5), opac=[math.log((1 / 300) / (1 - 1 / 300))], bg=(0.3, 0.3, 0.3))
    out = oracle_lib.Oracle(sc).forward()
    assert (out["ncontrib"][0] == 0).all()
    assert np.all(out["rgb"][0] == 0.3)
    assert np.all(out["alpha"][0] == 0.0)


def test_depth_ties_by_index(oracle_lib):
    # three identical Gaussians at the same depth: keys equal, values ascending
    sh = np.array([[[1.0, 0, 0]], [[0, 1.0, 0]], [[0, 0, 1.0]]], np.float32)
    sc = _one([[0, 0, 4.0]] * 3, math.log(0.5), opac=[0.0] * 3, sh=sh)
    o = oracle_lib.Oracle(sc)
    keys, vals, ranges = o.lists()
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        assert list(vals[s:e]) == sorted(vals[s:e])
    out = o.forward()
    # first-listed (index 0, red) dominates the composite at the centre
    px = (31, 31)
    rgb = [out["rgb"][0][ch][px] for ch in range(3)]
    assert rgb[0] > rgb[1] > rgb[2]


def test_empty_and_all_culled(oracle_lib):
    bg = (0.2, 0.4, 0.6)
    sc = _one([[0, 0, 0.1], [0, 0, -3.0]], math.log(0.5), bg=bg)   # both behind the near plane
    o = oracle_lib.Oracle(sc)
    assert (o.mirror()["flags"] & 1).all()
    keys, vals, ranges = o.lists()
    assert keys.size == 0 and (ranges == 0).all()
    out = o.forward()
    for ch in range(3):
        assert np.all(out["rgb"][0][ch] == bg[ch])
    assert np.all(out["depth"][0] == 0) and np.all(out["ncontrib"][0] == 0)


# ---------------------------------------------------------------------------
# tiling, keys and ranges vs brute force
# ---------------------------------------------------------------------------

def _small_multi_view(seed=7, n=300, degree=3, tile=(16, 16), ragged=True):
    rng = np.random.default_rng(seed)
    w1, h1 = (70, 45) if ragged else (64, 48)
    views = [pinhole(w1, h1, f=60.0),
             pinhole(48, 40, f=50.0, viewmat=look_from([0.1, -0.05, -0.3], yaw_deg=8.0, pitch_deg=-4.0)),
             pinhole(33, 31, f=40.0, viewmat=look_from([-0.2, 0.1, 0.2], yaw_deg=-10.0),
                     subset=np.sort(rng.choice(n, n // 2, replace=False)).astype(np.uint32))]
    return scenes.random_scene(seed, n, views, degree, tile=tile, bg=(0.1, 0.2, 0.3))


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
def test_keys_ranges_invariants(oracle_lib, tile):
    sc = _small_multi_view(tile=tile)
    o = oracle_lib.Oracle(sc)
    m = o.mirror()
    keys, vals, ranges = o.lists()
    # the lists are the tile rectangles exactly: one entry per tile of each rectangle
    M = int(keys.size)
    assert 0 < M == int(m["tiles"].astype(np.int64).sum())
    # (key, value) strictly increasing
    k = keys.astype(np.uint64)
    assert np.all((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (vals[1:] > vals[:-1])))
    # ranges partition [0, M) in tile order
    nonempty = ranges[:, 1] > ranges[:, 0]
    assert (ranges[~nonempty] == 0).all()
    r = ranges[nonempty]
    assert r[0, 0] == 0 and r[-1, 1] == M and np.all(r[1:, 0] == r[:-1, 1])
    # every key lies in its record's rectangle and carries its depth bits
    tiles_of_key = (k >> np.uint64(32)).astype(np.int64)
    for i in range(M):
        rec = int(vals[i])
        v = int(np.searchsorted(o.rec_base, rec, side="right") - 1)
        t = tiles_of_key[i] - o.tile_base[v]
        TX = o.tiles_xy[v][0]
        tx, ty = t % TX, t // TX
        x0, y0, x1, y1 = m["rect"][rec]
        assert x0 <= tx < x1 and y0 <= ty < y1
        assert int(k[i] & np.uint64(0xFFFFFFFF)) == int(m["zbits"][rec])


def test_tiled_equals_brute_force(oracle_lib):
    sc = _small_multi_view()
    o = oracle_lib.Oracle(sc)
    a = o.forward()
    b = o.forward(brute=1)
    for key in ("rgb", "depth", "alpha", "tfinal", "ncontrib", "nexam"):
        for x, y in zip(a[key], b[key]):
            assert np.array_equal(x, y), key


def test_low_opacity_brute_force_over_all_gaussians(oracle_lib):
    # The tile rectangle's upper edge, trunc((u + r + B - 1) / B), can lie half a
    # pixel inside the radius r = ceil(3 sqrt(lambda_max)).  Over lambda_max >= 0.3
    # the largest exp(-d^2 / (2 lambda)) at d = r - 1/2 is below 0.08, so with
    # sigma < 0.049 every truncated tail is below 1/255 and the rectangle test
    # drops nothing: compositing over all Gaussians equals the tiled result.
    sc = _small_multi_view(seed=9)
    sc.opacity_logits = np.minimum(sc.opacity_logits, -3.5).astype(np.float32)
    o = oracle_lib.Oracle(sc)
    a = o.forward()
    b = o.forward(brute=2)
    for key in ("rgb", "depth", "alpha", "tfinal"):
        for x, y in zip(a[key], b[key]):
            assert np.allclose(x, y, atol=1e-12), key


# ---------------------------------------------------------------------------
# binary32 decisions vs double precision
# ---------------------------------------------------------------------------

def test_mirror_agrees_with_fp64(oracle_lib):
    sc = scenes.small_box()
    o = oracle_lib.Oracle(sc)
    m, r = o.mirror(), o.rec64()
    vis = (m["flags"] & 1) == 0
    assert vis.sum() > 9000
    bl = m["blend"][vis].astype(np.float64)
    assert np.allclose(bl[:, 0], r[vis, 0], rtol=1e-6, atol=1e-4)
    assert np.allclose(bl[:, 1], r[vis, 1], rtol=1e-6, atol=1e-4)
    l2e = math.log2(math.e)
    assert np.allclose(bl[:, 2], -0.5 * l2e * r[vis, 2], rtol=2e-4, atol=1e-7)
    assert np.allclose(bl[:, 4], -0.5 * l2e * r[vis, 4], rtol=2e-4, atol=1e-7)
    assert np.allclose(bl[:, 5], r[vis, 5], rtol=1e-6)
    assert np.allclose(m["colour"][vis], r[vis, 6:9], atol=1e-6)
    # the decisions may differ only on near-threshold items, fewer than 1e-5 of
    # them: radius and rectangle per record, the compositing decisions per
    # examined (pixel, entry) pair (a pixel whose contributor count differs
    # counts as one disagreeing item); the disagreeing items are listed on failure
    r64 = o.rect64()
    same = np.all(r64[:, :5] == np.c_[m["radius"], m["rect"]], axis=1) | ~vis
    assert (~same).sum() <= int(1e-5 * vis.sum()), np.nonzero(~same)[0][:20]
    a = o.forward()
    b = o.forward(decide64=1)
    diff = a["ncontrib"][0] != b["ncontrib"][0]
    items = int(a["nexam"][0].sum())
    assert items > 1_000_000
    assert diff.sum() <= 1e-5 * items, list(zip(*np.nonzero(diff)))[:20]
    assert np.abs(a["rgb"][0] - b["rgb"][0]).max() < 5e-2


# ---------------------------------------------------------------------------
# analytic adjoint vs central finite differences of the FP64 forward
# ---------------------------------------------------------------------------

def _loss_weights(o, seed):
    rng = np.random.default_rng(seed)
    blocks = o.full_blocks()
    w_rgb = [rng.standard_normal((3, b[4], b[3])) for b in blocks]
    w_d = [0.1 * rng.standard_normal((b[4], b[3])) for b in blocks]
    w_a = [rng.standard_normal((b[4], b[3])) for b in blocks]
    return w_rgb, w_d, w_a


def _loss(o, w):
    out = o.forward()
    w_rgb, w_d, w_a = w
    return sum(float((a * b).sum()) for a, b in zip(out["rgb"], w_rgb)) + \
        sum(float((a * b).sum()) for a, b in zip(out["depth"], w_d)) + \
        sum(float((a * b).sum()) for a, b in zip(out["alpha"], w_a))


def _fd_scene(seed=11):
    views = [pinhole(40, 36, f=40.0),
             pinhole(34, 30, f=36.0, viewmat=look_from([0.15, -0.1, -0.4], yaw_deg=12.0, pitch_deg=5.0, roll_deg=3.0))]
    sc = scenes.random_scene(seed, 14, views, 3, z_range=(2.0, 4.0), xy_half=1.0,
                             log_scale_range=(-2.2, -1.2), bg=(0.2, 0.1, 0.3))
    # one Gaussian far off to the side so that the frustum guard clamps
    sc.means[0] = np.array([3.5, 0.2, 2.5], np.float32)
    sc.log_scales[0] = np.log(np.array([0.4, 0.3, 0.35], np.float32))
    return sc


def test_adjoint_matches_finite_differences(oracle_lib):
    sc = _fd_scene()
    o = oracle_lib.Oracle(sc)
    assert (o.mirror()["flags"] & 6).any(), "guard clamp not exercised"
    w = _loss_weights(o, 5)
    g = o.backward(w[0], w[1], w[2])
    base = {k: np.asarray(getattr(sc, k if k != "sh" else "sh"), np.float64).copy()
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    worst = 0.0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = base[name]
        flat = arr.reshape(-1)
        ana = g[name].reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            p = {k: v.copy() for k, v in base.items()}
            p[name].reshape(-1)[i] += h
            o.set_values(params64=p)
            lp = _loss(o, w)
            p[name].reshape(-1)[i] -= 2 * h
            o.set_values(params64=p)
            lm = _loss(o, w)
            fd = (lp - lm) / (2 * h)
            err = abs(fd - ana[i]) / max(1e-3, abs(fd), abs(ana[i]))
            worst = max(worst, err)
            assert err < 1e-5, (name, i, fd, ana[i])
    o.set_values()
    assert worst < 1e-5


def _se3_exp(delta):
    rho, om = np.asarray(delta[:3], np.float64), np.asarray(delta[3:], np.float64)
    th = np.linalg.norm(om)
    K = np.array([[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]])
    if th < 1e-12:
        R = np.eye(3) + K
        V = np.eye(3)
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def test_pose_gradient_matches_finite_differences(oracle_lib):
    sc = _fd_scene(seed=13)
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 6)
    vm = np.stack([v.viewmat.astype(np.float64) for v in sc.views])
    campos = np.stack([-(m[:3, :3].T @ m[:3, 3]) for m in vm])
    o.set_values(viewmats64=vm, campos64=campos)
    g = o.backward(w[0], w[1], w[2])
    for v in range(len(sc.views)):
        for k in range(6):
            h = 1e-6
            d = np.zeros(6); d[k] = h
            vp = vm.copy(); vp[v] = _se3_exp(d) @ vm[v]
            o.set_values(viewmats64=vp, campos64=campos)
            lp = _loss(o, w)
            d[k] = -h
            vp = vm.copy(); vp[v] = _se3_exp(d) @ vm[v]
            o.set_values(viewmats64=vp, campos64=campos)
            lm = _loss(o, w)
            fd = (lp - lm) / (2 * h)
            ana = g["pose"][v, k]
            assert abs(fd - ana) <= 1e-5 * max(1e-2, abs(fd), abs(ana)), (v, k, fd, ana)
    o.set_values()


def test_pose_translation_equals_summed_mean_gradient(oracle_lib):
    # degree 0: moving every Gaussian by d equals moving the camera by -R d, so
    # sum_g dL/dmu_g = R^T dL/drho for a single view
    views = [pinhole(40, 36, f=40.0, viewmat=look_from([0.1, 0.2, -0.3], yaw_deg=15.0, pitch_deg=-5.0))]
    sc = scenes.random_scene(17, 20, views, 0, z_range=(2.0, 4.0), xy_half=1.0, log_scale_range=(-2.2, -1.2))
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 7)
    g = o.backward(w[0], w[1], w[2])
    R = sc.views[0].viewmat[:3, :3].astype(np.float64)
    assert np.allclose(g["means"].sum(0), R.T @ g["pose"][0, :3], rtol=1e-9, atol=1e-12)


def test_isotropic_gaussian_has_no_rotation_gradient(oracle_lib):
    views = [pinhole(40, 36, f=40.0)]
    sc = scenes.random_scene(19, 10, views, 2, z_range=(2.0, 4.0), xy_half=1.0, log_scale_range=(-2.0, -1.5))
    sc.log_scales[:] = sc.log_scales[:, :1]
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 8)
    g = o.backward(w[0], w[1], w[2])
    assert np.abs(g["quats"]).max() < 1e-12 * max(1.0, np.abs(g["means"]).max())


def test_sh_gradient_closed_form(oracle_lib):
    # dL/dk_i = sum over views of Y_i(d_v) * dL/dcolour_v (unclamped channels)
    sc = _small_multi_view(seed=21, n=40)
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 9)
    g = o.backward(w[0], w[1], w[2], want_grec=True)
    m = o.mirror()
    exp = np.zeros_like(g["sh"])
    for v, view in enumerate(sc.views):
        vm = view.viewmat.astype(np.float64)
        cam = -(vm[:3, :3].T @ vm[:3, 3])
        for j in range(int(o.counts[v])):
            r = int(o.rec_base[v]) + j
            if m["flags"][r] & 1:
                continue
            gi = j if view.subset is None else int(view.subset[j])
            d = sc.means[gi].astype(np.float64) - cam
            b, _ = oracle_lib.sh_basis_f64(3, d / np.linalg.norm(d))
            gc = g["grec"][r, 6:9] * np.array([0.0 if m["flags"][r] & (32 << ch) else 1.0 for ch in range(3)])
            exp[gi] += np.outer(b, gc)
    assert np.allclose(g["sh"], exp, atol=1e-12)


def test_restricted_lists_equal_full_list_slices(oracle_lib):
    sc = _small_multi_view(seed=23)
    full = oracle_lib.Oracle(sc)
    keys, vals, ranges = full.lists()
    part = oracle_lib.Oracle(sc)
    rng = np.random.default_rng(3)
    tiles = sorted(set(int(t) for t in rng.integers(0, part.n_tiles, 9)))
    pk, pv, pr = part.restrict_tiles(tiles)
    for t in range(part.n_tiles):
        if t in tiles:
            a, b = ranges[t]
            c, d = pr[t]
            assert np.array_equal(keys[a:b], pk[c:d]) and np.array_equal(vals[a:b], pv[c:d])
        else:
            assert pr[t][0] == 0 and pr[t][1] == 0


def _anisotropic_scene(seed, n=400, opacity_shift=0.0):
    """Elongated, rotated Gaussians of mixed opacity (the case tile culling
    removes most from), on two views with ragged edges."""
    rng = np.random.default_rng(seed)
    views = [pinhole(70, 45, f=60.0),
             pinhole(48, 40, f=50.0, viewmat=look_from([0.1, -0.05, -0.3], yaw_deg=8.0, pitch_deg=-4.0))]
    sc = scenes.random_scene(seed, n, views, 3, tile=(16, 16), bg=(0.1, 0.2, 0.3))
    ls = np.log(np.exp(sc.log_scales) * np.array([6.0, 0.3, 1.0])).astype(np.float32)
    op = (sc.opacity_logits + opacity_shift + rng.normal(0, 1.5, sc.n)).astype(np.float32)
    return scenes.Scene(sc.name, sc.means, ls, sc.quats, op, sc.sh, sc.sh_degree, views, tile=sc.tile, bg=sc.bg,
                        target_seed=sc.target_seed)


def _with_lists(o, keys, vals, ranges):
    """Make later forward() calls of oracle o walk the given lists."""
    o._lists = (keys, vals, ranges, np.ascontiguousarray(vals if vals.size else np.zeros(1, np.uint32)))
    return o


def _filtered(o, keep):
    """o's lists with only the entries where keep is true (order kept)."""
    keys, vals, ranges = o.lists()
    k2, v2 = keys[keep], vals[keep]
    tiles = (k2 >> np.uint64(32)).astype(np.int64)
    r2 = np.zeros_like(ranges)
    if k2.size:
        starts = np.searchsorted(tiles, np.arange(ranges.shape[0]), side="left")
        ends = np.searchsorted(tiles, np.arange(ranges.shape[0]), side="right")
        ne = ends > starts
        r2[ne, 0], r2[ne, 1] = starts[ne], ends[ne]
    return np.ascontiguousarray(k2), np.ascontiguousarray(v2), r2


@pytest.mark.parametrize("seed,shift", [(41, 0.0), (42, -3.0), (43, 2.0)])
def test_lists_without_unreached_entries_composite_the_same(oracle_lib, seed, shift):
    """Entries that pass the alpha test at no pixel of their tile (reach 0)
    are inert: lists without them composite the same records in the same
    order, so every image, T_final, the blended count and the stop record of
    every pixel are identical, and each pixel's last composited record is
    the same record."""
    sc = _anisotropic_scene(seed, opacity_shift=shift)
    a = oracle_lib.Oracle(sc)
    reach = a.reach().astype(bool)
    keys, vals, ranges = a.lists()
    assert 0 < reach.sum() < reach.size            # thin Gaussians: many entries reach nothing
    fa = a.forward()
    b = _with_lists(oracle_lib.Oracle(sc), *_filtered(a, reach))
    fb = b.forward()
    for key in ("rgb", "depth", "alpha", "tfinal", "nblend", "stoprec"):
        for x, y in zip(fa[key], fb[key]):
            assert np.array_equal(x, y), key
    _, vb, rb = b.lists()
    for v, (x, y) in enumerate(zip(fa["ncontrib"], fb["ncontrib"])):
        h, w = x.shape
        ys, xs = np.mgrid[0:h, 0:w]
        t = a.tile_base[v] + (ys // sc.tile[1]) * a.tiles_xy[v][0] + xs // sc.tile[0]
        xi, yi = x.astype(np.int64), y.astype(np.int64)
        last_a = np.where(xi > 0, vals[np.maximum(ranges[t, 0].astype(np.int64) + xi - 1, 0)].astype(np.int64), -1)
        last_b = np.where(yi > 0, vb[np.maximum(rb[t, 0].astype(np.int64) + yi - 1, 0)].astype(np.int64), -1)
        assert np.array_equal(last_a, last_b)


def test_dropping_a_reached_entry_changes_the_walk(oracle_lib):
    """Each entry with reach 1 that composites or stops a pixel cannot be
    removed: the lists without it change that pixel (checked for a sample
    of such entries, one removal at a time)."""
    sc = _anisotropic_scene(45, n=120)
    a = oracle_lib.Oracle(sc)
    reach = a.reach().astype(bool)
    keys, vals, ranges = a.lists()
    fa = a.forward()
    rng = np.random.default_rng(0)
    idx = rng.choice(np.nonzero(reach)[0], 12, replace=False)
    changed = 0
    for k in idx:
        keep = np.ones(keys.size, bool)
        keep[k] = False
        fb = _with_lists(oracle_lib.Oracle(sc), *_filtered(a, keep)).forward()
        changed += any(not np.array_equal(x, y) for key in ("tfinal", "nblend", "stoprec")
                       for x, y in zip(fa[key], fb[key]))
    # an entry can reach 1/255 only behind pixels that stopped earlier; most change the image
    assert changed >= 9


def test_reach_of_an_isotropic_gaussian_closed_form(oracle_lib):
    """A single isotropic Gaussian reaches alpha >= 1/255 within the disc
    d^2 <= 2 a ln(255 sigma), a = (f s / z)^2 + 0.3: a tile is reached iff its
    nearest in-view pixel centre lies in that disc (tiles within 1e-3 px of
    the circle are not judged)."""
    f, z, s, op = 64.0, 4.0, 0.35, -2.0
    sc = _one([[0.13, -0.07, z]], math.log(s), opac=[op], views=[pinhole(96, 80, f=f)], tile=(4, 4))
    o = oracle_lib.Oracle(sc)
    reach = o.reach()
    keys, vals, ranges = o.lists()
    assert keys.size == reach.size > 0
    m = o.mirror()
    u, v = float(m["blend"][0, 0]), float(m["blend"][0, 1])
    a = (f * _s(s) / z) ** 2 + 0.3
    R2 = 2 * a * math.log(255 * _sigmoid(op))
    TX = o.tiles_xy[0][0]
    judged = 0
    for i, key in enumerate(keys):
        t = int(key >> np.uint64(32))
        tx, ty = t % TX, t // TX
        xs = np.arange(tx * 4, min(tx * 4 + 4, 96)) + 0.5
        ys = np.arange(ty * 4, min(ty * 4 + 4, 80)) + 0.5
        d2 = ((xs[None, :] - u) ** 2 + (ys[:, None] - v) ** 2).min()
        if abs(math.sqrt(d2) - math.sqrt(R2)) < 1e-3:
            continue
        judged += 1
        assert bool(reach[i]) == (d2 <= R2), (tx, ty, d2, R2)
    assert judged > 40 and 0 < reach.sum() < reach.size


def test_stop_record_is_the_entry_that_ends_the_walk(oracle_lib):
    """stoprec names the entry whose alpha would take T below 1e-4: opaque
    on-axis Gaussians clamp at alpha 0.99, so the binary32 sequence
    T = 1, 0.01, ... decides which entry stops the centre pixel; a pixel far
    from the centre does not stop."""
    zs = [3.0, 4.0, 5.0, 6.0]
    sc = _one([[0, 0, z] for z in zs], math.log(0.6), opac=[12.0] * len(zs))
    out = oracle_lib.Oracle(sc).forward()
    sr, nc = out["stoprec"][0], out["ncontrib"][0]
    T, k_stop = np.float32(1.0), None
    for k in range(len(zs)):
        Tn = np.float32(T * np.float32(np.float32(1.0) - np.float32(0.99)))
        if Tn < np.float32(1e-4):
            k_stop = k
            break
        T = Tn
    assert k_stop is not None
    assert sr[31, 31] == k_stop and nc[31, 31] == k_stop
    assert sr[0, 0] == 0xFFFFFFFF


def test_focal_gradient_matches_finite_differences(oracle_lib):
    """dL/dfx, dL/dfy per view against central differences of the value path
    (the scene has a Gaussian under the frustum guard, where fx x~ does not
    depend on fx)."""
    sc = _fd_scene(seed=23)
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 8)
    intr = np.array([[v.fx, v.fy, v.cx, v.cy] for v in sc.views], np.float64)
    o.set_values(intr64=intr)
    g = o.backward(w[0], w[1], w[2])
    for v in range(len(sc.views)):
        for k in range(2):
            h = 1e-4 * intr[v, k]
            ip = intr.copy(); ip[v, k] += h
            o.set_values(intr64=ip)
            lp = _loss(o, w)
            ip[v, k] -= 2 * h
            o.set_values(intr64=ip)
            lm = _loss(o, w)
            fd = (lp - lm) / (2 * h)
            ana = g["focal"][v, k]
            assert abs(fd - ana) <= 1e-5 * max(1e-2, abs(fd), abs(ana)), (v, k, fd, ana)
    o.set_values()


def _rig_scene(seed=29):
    """Two keyframes of a two-camera rig: V_i = A_c V_m(k)."""
    central = [look_from([0.0, 0.0, 0.0]), look_from([0.2, -0.05, 0.3], yaw_deg=6.0, pitch_deg=-3.0)]
    A = [np.eye(4), look_from([0.12, 0.02, 0.05], yaw_deg=-9.0, roll_deg=2.0)]
    views, kf, cam, rel = [], [], [], []
    for k, Vm in enumerate(central):
        for c, Ac in enumerate(A):
            views.append(pinhole(40, 34, f=38.0 + 2 * c, viewmat=(Ac.astype(np.float64) @ Vm.astype(np.float64))))
            kf.append(k); cam.append(c); rel.append(np.asarray(Ac, np.float64)[:3, :])
    sc = scenes.random_scene(seed, 16, views, 2, z_range=(2.0, 4.0), xy_half=1.0, log_scale_range=(-2.2, -1.2),
                             bg=(0.2, 0.1, 0.3))
    return sc, [np.asarray(V, np.float64) for V in central], np.asarray(A, np.float64), kf, cam, np.stack(rel)


def test_rig_chain_matches_finite_differences(oracle_lib):
    """The central pose of each keyframe and the focal length of each rig
    camera: the chain of the per-view gradients against central differences
    of the loss under the rig parametrisation."""
    sc, central, A, kf, cam, rel = _rig_scene()
    o = oracle_lib.Oracle(sc)
    w = _loss_weights(o, 9)
    vm = np.stack([v.viewmat.astype(np.float64) for v in sc.views])
    campos = np.stack([-(m[:3, :3].T @ m[:3, 3]) for m in vm])
    intr = np.array([[v.fx, v.fy, v.cx, v.cy] for v in sc.views], np.float64)
    o.set_values(viewmats64=vm, campos64=campos, intr64=intr)
    g = o.backward(w[0], w[1], w[2])
    ch = oracle_lib.rig_chain(g["pose"], kf, rel, 2, focal_grads=g["focal"], camera_of_view=cam, n_cameras=2)
    for k in range(2):
        for j in range(6):
            h = 1e-6
            vals = []
            for sgn in (1, -1):
                d = np.zeros(6); d[j] = sgn * h
                Vm = _se3_exp(d) @ central[k]
                vp = vm.copy()
                for i in range(len(sc.views)):
                    if kf[i] == k:
                        vp[i] = A[cam[i]] @ Vm
                o.set_values(viewmats64=vp, campos64=campos, intr64=intr)
                vals.append(_loss(o, w))
            fd = (vals[0] - vals[1]) / (2 * h)
            ana = ch["central"][k, j]
            assert abs(fd - ana) <= 1e-5 * max(1e-2, abs(fd), abs(ana)), (k, j, fd, ana)
    for c in range(2):
        for j in range(2):
            h = 1e-4 * intr[0, j]
            vals = []
            for sgn in (1, -1):
                ip = intr.copy()
                for i in range(len(sc.views)):
                    if cam[i] == c:
                        ip[i, j] += sgn * h
                o.set_values(viewmats64=vm, campos64=campos, intr64=ip)
                vals.append(_loss(o, w))
            fd = (vals[0] - vals[1]) / (2 * h)
            ana = ch["camera_focal"][c, j]
            assert abs(fd - ana) <= 1e-5 * max(1e-2, abs(fd), abs(ana)), (c, j, fd, ana)
    # the relative transform of the non-central camera, A_1 <- exp(delta^) A_1
    for j in range(6):
        h = 1e-6
        vals = []
        for sgn in (1, -1):
            d = np.zeros(6); d[j] = sgn * h
            A1 = _se3_exp(d) @ A[1]
            vp = vm.copy()
            for i in range(len(sc.views)):
                if cam[i] == 1:
                    vp[i] = A1 @ central[kf[i]]
            o.set_values(viewmats64=vp, campos64=campos, intr64=intr)
            vals.append(_loss(o, w))
        fd = (vals[0] - vals[1]) / (2 * h)
        ana = ch["camera_rel"][1, j]
        assert abs(fd - ana) <= 1e-5 * max(1e-2, abs(fd), abs(ana)), (j, fd, ana)
    o.set_values()
