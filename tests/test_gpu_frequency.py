"""GPU parity of the frequency-based scheduler (Sec. 3.3, Eq. 9-12) with the
oracle: X(I) per image within a norm-wise FP32 FFT error bound of the FP64
value, and the scheduler's decisions (r, r', level-up, sampled frames)
bit-exact against the oracle's binary32 mirror fed the same X values.

Tolerance of X: a Stockham FFT in binary32 has norm-wise error
||F^ - F||_2 <= g ||F||_2 with g ~ (7 log2 N + 2 sum of direct-pass radices) eps
(Higham, Accuracy and Stability of Numerical Algorithms, Thm. 24.2, with the
direct radix-p passes counted as p-term sums), and
|X^ - X| <= sum_f |F^_f - F_f| <= sqrt(N_f) ||F^ - F||_2; the test allows
10 (log2 N + sum p) eps sqrt(N_f) ||F||_2 / X, relative, per image."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300._lib import GsrError  # noqa: E402

import _parity as P  # noqa: E402

EPS = 2.0 ** -24


def _direct_primes(n):
    out = 0
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    p = 7
    while n > 1:
        while n % p == 0:
            out += p
            n //= p
        p += 2
    return out


def _bound(img, factor):
    a = oracle.box_downsample(img, factor)
    h, w = a.shape[1:]
    if h == 0 or w == 0:
        return 0.0, 0.0
    F = np.fft.fft2(a, axes=(1, 2))
    mag = np.sqrt((np.abs(F) ** 2).sum(0))
    x = float(mag.sum())
    norm = float(np.sqrt((mag ** 2).sum()))
    g = 10.0 * (math.log2(max(h * w, 2)) + _direct_primes(h) + _direct_primes(w)) * EPS
    return x, max(1e-6, g * math.sqrt(h * w) * norm / max(x, 1e-300))


def _raster():
    from paper_2512_08498_gb300.rasterizer import Rasterizer
    return Rasterizer(device=P.device())


def _check(r, imgs, factors):
    dev = P.device()
    ts = [torch.from_numpy(np.ascontiguousarray(i, np.float32)).to(dev) for i in imgs]
    x = r.dft_energy([(t, i.shape[2], i.shape[1], f) for t, i, f in zip(ts, imgs, factors)]).cpu().numpy()
    for k, (img, f) in enumerate(zip(imgs, factors)):
        exp, tol = _bound(np.asarray(img, np.float32).astype(np.float64), f)
        if exp == 0.0:
            assert x[k] == 0.0
        else:
            assert abs(x[k] - exp) <= tol * exp, (k, img.shape, f, x[k], exp, tol)
    return x


SIZES = [(1, 1), (1, 2), (3, 1), (5, 7), (8, 8), (64, 48), (100, 75), (49, 121), (97, 112), (13, 250), (45, 36),
         (256, 256), (27, 125), (2, 4096)]


def test_sizes_and_radices():
    rng = np.random.default_rng(1)
    imgs = [rng.random((3, h, w)) for h, w in SIZES]
    _check(_raster(), imgs, [1] * len(imgs))


@pytest.mark.parametrize("factor", [2, 3, 8])
def test_box_downsampled_levels(factor):
    rng = np.random.default_rng(factor)
    imgs = [rng.random((3, h, w)) for h, w in [(90, 160), (35, 47), (9, 17), (8, 8), (2, 30)]]
    _check(_raster(), imgs, [factor] * len(imgs))


def test_closed_forms_on_power_of_two_sizes():
    """Radix-4/2 sizes transform constants exactly: X = h w ||c||; an impulse
    gives h w ||a||."""
    h, w = 64, 128
    c = np.array([0.25, 0.5, 0.75])
    const = np.broadcast_to(c[:, None, None], (3, h, w)).astype(np.float32)
    a = np.array([1.0, -2.0, 0.5])
    imp = np.zeros((3, h, w), np.float32)
    imp[:, 5, 77] = a
    x = _check(_raster(), [const, imp], [1, 1])
    assert x[0] == pytest.approx(h * w * np.linalg.norm(c), rel=1e-6)
    assert x[1] == pytest.approx(h * w * np.linalg.norm(a), rel=1e-6)


def test_many_images_and_lengths_span_several_launch_tables():
    """More images than one launch table holds and more distinct lengths
    than its plan table: the batch is split, results unchanged."""
    rng = np.random.default_rng(9)
    imgs = [rng.random((3, 3 + (k % 37), 4 + (k * 7) % 41)) for k in range(230)]
    _check(_raster(), imgs, [1] * len(imgs))


def test_empty_and_too_large_images():
    r = _raster()
    dev = P.device()
    t = torch.rand(3 * 5 * 7, device=dev)
    x = r.dft_energy([(t, 7, 5, 8), (t, 7, 5, 1), (t, 0, 0, 1)]).cpu().numpy()
    assert x[0] == 0.0 and x[1] > 0 and x[2] == 0.0
    big = torch.empty(3 * 4097, device=dev)
    with pytest.raises(GsrError):
        r.dft_energy([(big, 4097, 1, 1)])
    with pytest.raises(GsrError):
        r.dft_energy([(t, 7, 5, 0)])


def _schedule_compare(r, xg, xl, xr, tau, u):
    dev = P.device()
    tt = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(dev)
    got = r.frequency_schedule(tt(xg), tt(xr), x_gt_level=tt(xl), tau_f=tau, uniforms=tt(u))
    exp = oracle.frequency_schedule(xg, xl, xr, tau, u)
    assert np.array_equal(got["r"].cpu().numpy(), exp["r"], equal_nan=True)
    assert np.array_equal(got["r_level"].cpu().numpy(), exp["r_level"], equal_nan=True)
    assert np.array_equal(got["level_up"].cpu().numpy().astype(bool), exp["level_up"])
    assert np.array_equal(got["samples"].cpu().numpy(), exp["samples"])
    return exp


def test_schedule_on_rig_images_full_size():
    """The 6-camera 1600x900 rig: X of the seeded targets, of the targets at
    level 2 and of the rasterizer's renderings (every image against the
    oracle), then r, r', level-up and 4096 sampled frames bit-exact."""
    from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views
    sc = scenes.rig6()
    dev = P.device()
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg, device=dev)
    rgb, _, _, _ = r.forward(P.params_of(sc, dev), to_camera_views(sc.views, dev))
    gts = [t.astype(np.float32) for t in sc.targets()]
    offs = np.cumsum([0] + [3 * v.width * v.height for v in sc.views])
    rgb_h = rgb.cpu().numpy()
    rens = [rgb_h[offs[i]: offs[i + 1]].reshape(3, v.height, v.width) for i, v in enumerate(sc.views)]
    x = _check(r, gts + gts + rens, [1] * 6 + [2] * 6 + [1] * 6)
    u = np.random.default_rng(2).random(4096).astype(np.float32)
    exp = _schedule_compare(r, x[:6], x[6:12], x[12:], 2.0, u)
    assert (exp["r"] > 1).all()


def test_schedule_edge_cases():
    r = _raster()
    rng = np.random.default_rng(3)
    n = 300
    xg = rng.random(n).astype(np.float32) * 10
    xr = rng.random(n).astype(np.float32) * 5
    xl = (xr * rng.uniform(0.5, 3.5, n)).astype(np.float32)
    xr[7] = 0.0                   # empty rendering: r = inf, capped weight
    xg[9] = xr[9] = 0.0           # 0 / 0: NaN, weight 0
    xl[11] = np.float32(2.0) * xr[11]   # r' exactly tau: no level-up
    u = np.concatenate([rng.random(1000), [0.0, 1.0, np.nextafter(np.float32(1), np.float32(0))]]).astype(np.float32)
    _schedule_compare(r, xg, xl, xr, 2.0, u)
    # no positive weight: uniform over the frames
    z = np.zeros(5, np.float32)
    _schedule_compare(r, z, z, np.ones(5, np.float32), 2.0, np.linspace(0, 0.99, 11).astype(np.float32))
    with pytest.raises(GsrError):
        r.frequency_schedule(torch.zeros(4097, device=P.device()), torch.ones(4097, device=P.device()))
