"""Pins of the scheduler oracle (Sec. 3.3, Eq. 9-12): X(I) = sum over
frequencies of the channel norm of the unnormalised 2-D DFT, against a
brute-force DFT written out as sums, closed forms (constant, impulse and
plane-wave images), invariants (circular shifts, scaling, transposition,
channel order), the box downsampling, and the binary32 schedule decisions
on hand-worked cases."""
import math

import numpy as np
import pytest

import oracle


def _brute_x(img):
    """The DFT as its defining double sum, evaluated directly."""
    c, h, w = img.shape
    ys, xs = np.arange(h), np.arange(w)
    total = 0.0
    for i in range(h):
        for j in range(w):
            ph = np.exp(-2j * math.pi * (i * ys[:, None] / h + j * xs[None, :] / w))
            f = np.array([(img[ch] * ph).sum() for ch in range(c)])
            total += math.sqrt(float((np.abs(f) ** 2).sum()))
    return total


@pytest.mark.parametrize("h,w", [(1, 1), (1, 4), (3, 5), (6, 7), (8, 2)])
def test_matches_the_defining_sum(h, w):
    rng = np.random.default_rng(h * 10 + w)
    img = rng.random((3, h, w))
    assert oracle.dft_energy(img) == pytest.approx(_brute_x(img), rel=1e-12)


def test_constant_and_impulse_images():
    h, w = 9, 14
    c = np.array([0.2, 0.5, 0.7])
    img = np.broadcast_to(c[:, None, None], (3, h, w))
    # only the zero frequency: ||c|| h w
    assert oracle.dft_energy(img) == pytest.approx(h * w * np.linalg.norm(c), rel=1e-12)
    a = np.array([1.0, -2.0, 0.5])
    imp = np.zeros((3, h, w)); imp[:, 4, 11] = a
    # |DFT| = |a_c| at every frequency: h w ||a|| (a per-channel sum would give h w sum|a_c|)
    assert oracle.dft_energy(imp) == pytest.approx(h * w * np.linalg.norm(a), rel=1e-12)


def test_plane_wave():
    h, w = 12, 20
    yy, xx = np.mgrid[0:h, 0:w]
    wave = np.cos(2 * math.pi * (3 * xx / w + 2 * yy / h))
    c = np.array([0.5, 0.4, 0.3]); a = np.array([0.2, 0.1, -0.05])
    img = c[:, None, None] + a[:, None, None] * wave[None]
    # DC peak h w ||c||, two peaks of h w ||a|| / 2 at +-(2, 3)
    assert oracle.dft_energy(img) == pytest.approx(h * w * (np.linalg.norm(c) + np.linalg.norm(a)), rel=1e-12)


def test_invariants():
    rng = np.random.default_rng(3)
    img = rng.random((3, 10, 13))
    x = oracle.dft_energy(img)
    assert oracle.dft_energy(np.roll(img, (3, -5), axis=(1, 2))) == pytest.approx(x, rel=1e-12)
    assert oracle.dft_energy(-2.5 * img) == pytest.approx(2.5 * x, rel=1e-12)
    assert oracle.dft_energy(img.transpose(0, 2, 1)) == pytest.approx(x, rel=1e-12)
    assert oracle.dft_energy(img[[2, 0, 1]]) == pytest.approx(x, rel=1e-12)


def test_box_downsample():
    h, w = 9, 11
    yy, xx = np.mgrid[0:h, 0:w]
    checker = ((xx + yy) % 2).astype(np.float64)
    img = np.stack([checker, 1 - checker, 0.25 + 0 * checker])
    d = oracle.box_downsample(img, 2)
    assert d.shape == (3, 4, 5)
    assert np.allclose(d, np.array([0.5, 0.5, 0.25])[:, None, None])
    # factor 2 equals the transform of the downsampled image; factor 1 is the identity
    rng = np.random.default_rng(4)
    r = rng.random((3, 17, 23))
    assert oracle.dft_energy(r, 3) == pytest.approx(oracle.dft_energy(oracle.box_downsample(r, 3)), rel=1e-14)
    assert np.array_equal(oracle.box_downsample(r, 1), r)
    # each block mean by hand
    d3 = oracle.box_downsample(r, 3)
    assert d3.shape == (3, 5, 7)
    assert d3[1, 2, 4] == pytest.approx(r[1, 6:9, 12:15].mean(), rel=1e-15)
    assert oracle.dft_energy(np.zeros((3, 2, 2)), 3) == 0.0


def test_schedule_decisions_by_hand():
    xg = np.array([4.0, 6.0, 2.0], np.float32)
    xl = np.array([3.0, 2.0, 5.0], np.float32)
    xr = np.array([4.0, 2.0, 2.0], np.float32)
    s = oracle.frequency_schedule(xg, xl, xr, 2.0, [0.0, 0.19, 0.2, 0.21, 0.79, 0.8, 0.99])
    assert np.array_equal(s["r"], np.array([1.0, 3.0, 1.0], np.float32))
    assert np.array_equal(s["r_level"], np.array([0.75, 1.0, 2.5], np.float32))
    assert s["level_up"].tolist() == [True, True, False]
    # cumulative weights 1, 4, 5: t = 5u; first c > t
    assert s["samples"].tolist() == [0, 0, 1, 1, 1, 2, 2]


def test_schedule_degenerate_weights():
    # an empty rendering: r = inf, capped at 1e30, drawn almost surely
    s = oracle.frequency_schedule([1.0, 1.0], [1.0, 0.0], [0.0, 1.0], 2.0, [0.5, 0.999])
    assert np.isinf(s["r"][0]) and s["samples"].tolist() == [0, 0]
    assert s["level_up"].tolist() == [False, True]
    # 0 / 0: NaN weight 0, never level-up
    s = oracle.frequency_schedule([0.0, 3.0], [0.0, 3.0], [0.0, 1.0], 2.0, [0.0, 0.5])
    assert np.isnan(s["r"][0]) and s["samples"].tolist() == [1, 1] and s["level_up"].tolist() == [False, False]
    # all weights 0: uniform
    s = oracle.frequency_schedule([0.0, 0.0, 0.0], [0.0] * 3, [1.0] * 3, 2.0, [0.1, 0.5, 0.9])
    assert s["samples"].tolist() == [0, 1, 2]
    # the largest u below 1 still lands on a frame of positive weight (u total
    # rounds below the total); u = 1 itself falls back to the last such frame
    s = oracle.frequency_schedule([1.0, 1.0, 0.0], [1.0] * 3, [1.0] * 3, 2.0,
                                  [np.nextafter(np.float32(1), np.float32(0)), 1.0])
    assert s["samples"].tolist() == [1, 1]
