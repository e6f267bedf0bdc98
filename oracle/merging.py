"""Oracle of the inter-camera Gaussian merging (Sec. 3.2, Eq. 7-8).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.
Plain numpy plus the oracle's binary32 exponential; nothing shared with the
CUDA package.

When camera i of a rig adds Gaussians at its sampled pixels (the pixels of
Eq. 4-5 whose P_a exceeds tau_a, with scales S of Eq. 6), the Gaussians
already built from cameras 0 .. i-1 are reprojected into camera i and each is
paired with the sampled pixel its reprojection falls in, unless the depths
differ by more than tau_d.  Each sampled pixel with a non-empty group keeps
one primitive: the one with the smallest image-space scale (s' = S f / d' for
an existing Gaussian, s_i = S_i f / d_i = 1 / (2 sqrt(P(I_i))) for the sample,
Eq. 8 with Eq. 6); the others are dropped.  The kept primitive keeps its
attributes but takes the mean colour of the group (the SH DC coefficients;
a sample's own colour is its ground-truth pixel), and a kept sample is moved
to the mean depth of its group (its scale follows the depth, as Eq. 6 does).

Discrete decisions (pairing, depth test, which primitive is kept) are taken
in binary32 with the operation order written below; values are FP64.

Readings (the paper is silent or garbled on each): the pairing pixel is the
one containing the reprojected mean (u' = fx x/z + cx, pixel centres at
+1/2); d' and d_i are camera-space depths z; S of an existing Gaussian is its
largest scale; Eq. 7's 2 S f / d' is taken without the factor 2, so that the
two scales of a sample of Eq. 6 agree; ties keep the existing Gaussian of
lowest index; tau_d is a caller parameter (absolute, metres).

Parity with numbers printed by the paper is unpinned: the paper prints no
merging example.
"""
from __future__ import annotations

import numpy as np

SH_C0 = 0.28209479177387814     # Y_00 = 1 / (2 sqrt(pi))

INSERT, MERGED, REPLACES = 0, 1, 2          # sample actions
UNTOUCHED, REMOVED, KEPT = 0, 1, 2          # existing actions


def _f(x):
    return np.float32(x)


def merge(view, means, log_scales, sh_dc, sample_pixels, scale_map, depth_map, gt, tau_d=0.5, near=0.2,
          exp_f32=None) -> dict:
    """Merge camera i's samples with the existing Gaussians.

    view: fx, fy, cx, cy, width, height, viewmat (world-to-camera, 4x4).
    means, log_scales [N, 3]; sh_dc [N, 3] the degree-0 SH coefficients.
    sample_pixels [M] ascending pixel indices (y W + x) of camera i's samples;
    scale_map, depth_map [H, W] (S of Eq. 6, camera-space depth); gt [3, H, W].
    exp_f32: the binary32 exponential of the decision contract (scalar)."""
    if exp_f32 is None:
        from .oracle import exp_f32
    W, H = int(view.width), int(view.height)
    fx, fy, cx, cy = _f(view.fx), _f(view.fy), _f(view.cx), _f(view.cy)
    V32 = np.asarray(view.viewmat, np.float32)
    V64 = np.asarray(view.viewmat, np.float32).astype(np.float64)
    mu = np.asarray(means, np.float32).reshape(-1, 3)
    ls = np.asarray(log_scales, np.float32).reshape(-1, 3)
    dc_in = np.asarray(sh_dc, np.float64).reshape(-1, 3)
    sp = np.asarray(sample_pixels, np.int64).reshape(-1)
    Smap = np.asarray(scale_map, np.float32).reshape(-1)
    Dmap = np.asarray(depth_map, np.float32).reshape(-1)
    img = np.asarray(gt, np.float64).reshape(3, -1)
    N, M = mu.shape[0], sp.size
    tau = _f(tau_d)

    # ---- reprojection into camera i (binary32, left-to-right sums) ----
    def row(r):
        return ((V32[r, 0] * mu[:, 0] + V32[r, 1] * mu[:, 1]).astype(np.float32) + V32[r, 2] * mu[:, 2]).astype(
            np.float32) + V32[r, 3]
    x, y, z = (row(r).astype(np.float32) for r in range(3))
    front = z > _f(near)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = ((fx * (x / z).astype(np.float32)).astype(np.float32) + cx).astype(np.float32)
        v = ((fy * (y / z).astype(np.float32)).astype(np.float32) + cy).astype(np.float32)
    inside = front & (u >= 0) & (u < _f(W)) & (v >= 0) & (v < _f(H))
    slot_of_pixel = np.full(W * H, -1, np.int64)
    slot_of_pixel[sp] = np.arange(M)
    pair = np.full(N, -1, np.int64)
    s_ex = np.zeros(N, np.float32)
    for g in np.nonzero(inside)[0]:
        pix = int(np.floor(v[g])) * W + int(np.floor(u[g]))
        s = slot_of_pixel[pix]
        if s < 0:
            continue
        if not (abs(_f(z[g] - Dmap[pix])) <= tau):
            continue
        pair[g] = s
        S_g = _f(exp_f32(float(max(ls[g, 0], ls[g, 1], ls[g, 2]))))
        s_ex[g] = _f(_f(S_g * fx) / z[g])

    # ---- per sampled pixel: keep the smallest image-space scale ----
    z64 = (V64[2, :3] @ mu.astype(np.float64).T) + V64[2, 3] if N else np.zeros(0)
    s_act = np.full(M, INSERT, np.int32)
    e_act = np.full(N, UNTOUCHED, np.int32)
    e_dc = dc_in.copy()
    d_p = Dmap[sp].astype(np.float64)
    own_dc = ((img[:, sp] - 0.5) / SH_C0).T if M else np.zeros((0, 3))
    s_dc = own_dc.copy()
    s_depth = d_p.copy()
    groups = {}
    for g in np.nonzero(pair >= 0)[0]:
        groups.setdefault(int(pair[g]), []).append(int(g))
    for s, members in groups.items():
        best = min(members, key=lambda g: (float(s_ex[g]), g))
        pix = int(sp[s])
        s_new = _f(_f(Smap[pix] * fx) / Dmap[pix])
        mean_dc = (own_dc[s] + dc_in[members].sum(axis=0)) / (len(members) + 1)
        if s_new < s_ex[best]:
            s_act[s] = REPLACES
            s_dc[s] = mean_dc
            s_depth[s] = (d_p[s] + z64[members].sum()) / (len(members) + 1)
            e_act[members] = REMOVED
        else:
            s_act[s] = MERGED
            e_act[members] = REMOVED
            e_act[best] = KEPT
            e_dc[best] = mean_dc

    # ---- the samples as Gaussians: unprojected pixel centres, Eq. 6 scales ----
    px = (sp % W).astype(np.float64) + 0.5
    py = (sp // W).astype(np.float64) + 0.5
    cam = np.stack([(px - float(view.cx)) / float(view.fx) * s_depth,
                    (py - float(view.cy)) / float(view.fy) * s_depth, s_depth], axis=1) if M else np.zeros((0, 3))
    Rm, tv = V64[:3, :3], V64[:3, 3]
    s_means = (cam - tv) @ Rm                      # R^T (p - t), row vectors
    s_scale = Smap[sp].astype(np.float64) * s_depth / np.where(d_p > 0, d_p, 1.0)
    return {"sample_action": s_act, "sample_dc": s_dc, "sample_depth": s_depth, "sample_means": s_means,
            "sample_scale": s_scale, "existing_action": e_act, "existing_dc": e_dc, "pair": pair,
            "s_existing": s_ex}
