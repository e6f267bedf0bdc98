"""Pins of the oracle's insertion probability and scale initialisation
(Sec. 3.2, Eq. 4-6): P(I) = min(||LoG_sigma * I||, 1), P_a = max(P(I) - P(I~), 0),
insertion where P_a > tau_a, S = d / (2 sqrt(P(I)) f).  Each check compares the
oracle with something other than its own formula: closed forms of the
Laplacian of a Gaussian-blurred image, invariants of the kernel, special
images whose response is known."""
import math

import numpy as np
import pytest


def _view(h, w, fill):
    return np.broadcast_to(np.asarray(fill, np.float32)[:, None, None], (3, h, w)).copy()


def test_taps_zero_mean_symmetric_and_centre(oracle_lib):
    t32, t64 = oracle_lib.log_taps(1.0)
    assert t64.shape == (7, 7)
    assert abs(t64.sum()) < 1e-15
    assert np.allclose(t64, t64[::-1, :]) and np.allclose(t64, t64[:, ::-1]) and np.allclose(t64, t64.T)
    # continuous LoG at the origin, -2 s^2 / s^4 / (2 pi s^2) = -1/pi for s = 1, less the mean
    x = np.arange(-3, 4)
    q = x[None, :] ** 2 + x[:, None] ** 2
    raw = (q - 2.0) * np.exp(-q / 2.0) / (2 * math.pi)
    assert t64[3, 3] == pytest.approx(-1.0 / math.pi - raw.mean(), rel=1e-12)
    assert np.array_equal(t32, t64.astype(np.float32))
    # radius ceil(3 sigma)
    assert oracle_lib.log_taps(0.5)[1].shape == (5, 5)
    assert oracle_lib.log_taps(2.0)[1].shape == (13, 13)


def test_constant_and_ramp_images_respond_zero(oracle_lib):
    h, w = 23, 37
    d = np.full((h, w), 3.0, np.float32)
    const = _view(h, w, [0.3, 0.7, 0.1])
    out = oracle_lib.insertion(const, const, d, 100.0)
    assert np.abs(out["p_gt"]).max() < 1e-12 and not out["inserted"].any()
    # a linear ramp has zero Laplacian: the symmetric zero-mean kernel answers 0
    # away from the clamped border
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    # dyadic slopes: the ramp is exact in binary32
    ramp = np.stack([xx / 64 + yy / 32, 0.5 - yy / 128, xx / 256]).astype(np.float32)
    out = oracle_lib.insertion(ramp, const, d, 100.0)
    assert np.abs(out["p_gt"][3:-3, 3:-3]).max() < 1e-12


def test_impulse_response_is_the_kernel(oracle_lib):
    h, w = 15, 17
    img = np.zeros((3, h, w), np.float32)
    img[:, 7, 8] = 1.0
    zero = np.zeros_like(img)
    d = np.full((h, w), 5.0, np.float32)
    out = oracle_lib.insertion(img, zero, d, 100.0, tau_a=0.2)
    _, t64 = oracle_lib.log_taps(1.0)
    expect = np.zeros((h, w))
    expect[4:11, 5:12] = np.minimum(math.sqrt(3.0) * np.abs(t64), 1.0)
    assert np.allclose(out["p_gt"], expect, rtol=0, atol=1e-14)
    # rendering all black: P_a = P(I); inserted where above 0.2; scale from Eq. 6
    assert np.array_equal(out["p_a"], out["p_gt"])
    ins = out["inserted"]
    assert ins[7, 8] and ins.sum() == int((expect > 0.2).sum())
    pc = min(math.sqrt(3.0) * abs(t64[3, 3]), 1.0)
    assert out["scale"][7, 8] == pytest.approx(5.0 / (2.0 * math.sqrt(pc) * 100.0), rel=1e-12)
    assert (out["scale"][~ins] == 0).all()


def test_smooth_image_matches_the_continuous_laplacian_of_gaussian(oracle_lib):
    """For I = c + A sin(a x) sin(b y), LoG_s * I = -(a^2 + b^2) exp(-s^2 (a^2 + b^2) / 2)
    A sin(a x) sin(b y) exactly in the continuum; the sampled, truncated,
    zero-mean kernel agrees to ~1 % at these frequencies.  A wrong sign,
    dropped 2 s^2 term or normalisation fails by far more."""
    h, w = 64, 80
    a, b, A = 0.35, 0.25, 0.4
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    f = A * np.sin(a * xx) * np.sin(b * yy)
    img = np.stack([0.5 + f, 0.5 + 0.5 * f, 0.5 - f]).astype(np.float32)
    zero = np.zeros_like(img)
    out = oracle_lib.insertion(img, zero, np.ones((h, w), np.float32), 1.0)
    lap = -(a * a + b * b) * math.exp(-(a * a + b * b) / 2.0) * f
    norm = np.abs(lap) * math.sqrt(1.0 + 0.25 + 1.0)
    inner = (slice(4, -4), slice(4, -4))
    big = norm[inner] > 0.02
    rel = np.abs(out["p_gt"][inner][big] - norm[inner][big]) / norm[inner][big]
    assert rel.max() < 0.03


def test_clamp_at_one_and_equal_images(oracle_lib):
    h, w = 20, 20
    img = np.zeros((3, h, w), np.float32)
    img[:, 9, 9] = 4.0            # response sqrt(3) 4 / pi > 1 at the centre
    d = np.ones((h, w), np.float32)
    out = oracle_lib.insertion(img, img, d, 50.0)
    assert out["p_gt"][9, 9] == 1.0 and (out["p_gt"] <= 1.0).all()
    assert np.abs(out["p_a"]).max() == 0.0 and not out["inserted"].any()


def test_mirror_decision_agrees_with_double_away_from_the_threshold(oracle_lib):
    rng = np.random.default_rng(5)
    h, w = 45, 70
    gt = rng.random((3, h, w)).astype(np.float32)
    ren = np.clip(gt + rng.normal(0, 0.05, gt.shape), 0, 1).astype(np.float32)
    ren[:, 10:30, 20:50] = 0.5      # a flat, poorly reconstructed patch
    out = oracle_lib.insertion(gt, ren, np.full((h, w), 2.0, np.float32), 800.0)
    far = np.abs(out["p_a"] - 0.2) > 1e-5
    assert np.array_equal(out["inserted"][far], (out["p_a"] > 0.2)[far])
    assert out["inserted"].any() and not out["inserted"].all()
