"""Oracle of the frequency-based scheduler (Sec. 3.3, Eq. 9-12).

TEST INFRASTRUCTURE ONLY: imported by the tests and the CPU-baseline leg of
the benchmark, never by the product path.  Plain numpy; nothing shared with
the CUDA package.

* ``box_downsample``  the level-n ground truth I^n: the mean of each n x n
                      block, floor(H/n) x floor(W/n) (FP64);
* ``dft_energy``      X(I) = sum over all frequencies (i, j) of the Euclidean
                      norm, over the three colour channels, of the unnormalised
                      2-D DFT of each channel at (i, j) (Eq. 10, 11; FP64,
                      numpy's FFT as the DFT);
* ``frequency_schedule``  r = X(I) / X(I~) (Eq. 9), r' = X(I^n) / X(I~)
                      (Eq. 12), the level-up flags r' < tau_f, and frames drawn
                      with probability proportional to r by inverse CDF from
                      caller-supplied uniforms.  Those are discrete decisions:
                      they are taken in binary32, in the order written below,
                      from binary32 inputs.

Parity of the scheduler with numbers printed by the paper is unpinned: the
paper prints no value of X, r or r'.
"""
from __future__ import annotations

import numpy as np


def box_downsample(img, n: int) -> np.ndarray:
    """I^n for a planar image [C, H, W]: block means over n x n pixels, the
    trailing H mod n rows and W mod n columns dropped (FP64)."""
    a = np.asarray(img, np.float64)
    n = int(n)
    if n < 1:
        raise ValueError("factor must be >= 1")
    c, h, w = a.shape
    hn, wn = h // n, w // n
    a = a[:, : hn * n, : wn * n].reshape(c, hn, n, wn, n)
    return a.mean(axis=(2, 4))


def dft_energy(img, factor: int = 1) -> float:
    """Eq. 10: X(I) = sum_{i,j} || DFT(I)(i, j) ||_2 for a planar RGB image
    [3, H, W]; the DFT is the unnormalised 2-D transform of each channel and
    the norm is taken over the channels at each frequency."""
    a = box_downsample(img, factor) if int(factor) != 1 else np.asarray(img, np.float64)
    if a.shape[1] == 0 or a.shape[2] == 0:
        return 0.0
    F = np.fft.fft2(a, axes=(1, 2))
    return float(np.sqrt((np.abs(F) ** 2).sum(axis=0)).sum())


def _f32(x):
    return np.float32(x)


def frequency_schedule(x_gt, x_gt_level, x_rendered, tau_f: float, uniforms) -> dict:
    """Eq. 9 and 12 with the scheduler's two decisions, per frame f:

      r_f  = x_gt_f / x_rendered_f          (binary32 division)
      r'_f = x_gt_level_f / x_rendered_f
      level_up_f = r'_f < tau_f              (false for NaN)

    Sampling: the weight of frame f is r_f, with NaN taken as 0 and values
    above 1e30 as 1e30; c_f = c_{f-1} + w_f in binary32 from c_{-1} = 0.
    Sample s takes t = u_s * c_last (binary32) and draws the first f with
    c_f > t; if none has (only for u_s >= 1), the last frame of positive
    weight.  If every weight is 0, all frames weigh 1."""
    xg = np.asarray(x_gt, np.float32).reshape(-1)
    xl = np.asarray(x_gt_level, np.float32).reshape(-1)
    xr = np.asarray(x_rendered, np.float32).reshape(-1)
    n = xg.size
    tau = _f32(tau_f)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = (xg / xr).astype(np.float32)
        rl = (xl / xr).astype(np.float32)
    level_up = np.array([bool(v < tau) for v in rl], dtype=bool)
    w = np.empty(n, np.float32)
    for f in range(n):
        v = r[f]
        if np.isnan(v):
            v = _f32(0.0)
        elif v > _f32(1e30):
            v = _f32(1e30)
        w[f] = v
    if not (w > 0).any():
        w[:] = _f32(1.0)
    cum = np.empty(n, np.float32)
    acc = _f32(0.0)
    for f in range(n):
        acc = _f32(acc + w[f])
        cum[f] = acc
    last_pos = int(np.nonzero(w > 0)[0][-1]) if n else -1
    samples = []
    for u in np.asarray(uniforms, np.float32).reshape(-1):
        t = _f32(_f32(u) * cum[-1])
        pick = last_pos
        for f in range(n):
            if cum[f] > t:
                pick = f
                break
        samples.append(pick)
    return {"r": r, "r_level": rl, "level_up": level_up, "samples": np.asarray(samples, np.int32)}
