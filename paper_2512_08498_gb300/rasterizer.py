"""Python front end of libgsr: tensors in, tensors out, every step in CUDA.

PyTorch supplies device memory and the current stream; the rasterizer's work
(projection, sort, ranges, blending and their adjoints) runs in the kernels of
libgsr.so behind its C ABI.  ``rasterize`` is a ``torch.autograd.Function``
that returns RGB, depth and alpha images and gives gradients for the five
Gaussian parameter tensors and a per-view se(3) pose perturbation
(left-multiplied, ``V <- exp(delta^) V``; the SH direction is held constant
for the pose, the detachment the paper applies when it refines cameras,
Sec. 3.3).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L


@dataclass
class CameraView:
    """One pinhole view: intrinsics, row-major world-to-camera matrix, optional subset."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray                    # (4, 4) float32
    subset: Optional[torch.Tensor] = None  # int32/uint32 device tensor, ascending


def to_camera_views(views, device="cuda") -> List[CameraView]:
    """Convert seeded scene views (numpy subsets) to CameraView with device subsets."""
    out = []
    cache = {}
    for v in views:
        sub = None
        if v.subset is not None:
            key = id(v.subset)
            if key not in cache:
                cache[key] = torch.from_numpy(np.ascontiguousarray(v.subset.astype(np.int32))).to(device)
            sub = cache[key]
        out.append(CameraView(int(v.width), int(v.height), float(v.fx), float(v.fy), float(v.cx), float(v.cy),
                              np.asarray(v.viewmat, np.float32), sub))
    return out


def pixel_offsets(views: Sequence) -> List[int]:
    offs, o = [], 0
    for v in views:
        offs.append(o)
        o += int(v.width) * int(v.height)
    offs.append(o)
    return offs


def split_images(rgb: torch.Tensor, depth: torch.Tensor, alpha: torch.Tensor, views: Sequence):
    """Flat outputs -> per-view ([3,H,W], [H,W], [H,W]) views of the same storage."""
    offs = pixel_offsets(views)
    res = []
    for i, v in enumerate(views):
        a, b = offs[i], offs[i + 1]
        res.append((rgb[3 * a: 3 * b].view(3, v.height, v.width), depth[a:b].view(v.height, v.width),
                    alpha[a:b].view(v.height, v.width)))
    return res


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


_nonnull = {}


def _nonnull_ptr(dev) -> int:
    """A valid device address for an empty subset (NULL would mean 'all Gaussians')."""
    key = str(dev)
    if key not in _nonnull:
        _nonnull[key] = torch.zeros(4, dtype=torch.int32, device=dev)
    return _nonnull[key].data_ptr()


def _stream_ptr(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class _Saved:
    """Owner of a gsr_saved handle."""

    def __init__(self, raster: "Rasterizer"):
        self.lib = raster.lib
        self.raster = raster
        h = C.c_void_p()
        raster._check(self.lib.gsr_saved_create(raster.ctx, C.byref(h)))
        self.h = h

    def info(self) -> dict:
        i = L.SavedInfo()
        self.lib.gsr_saved_get_info(self.h, C.byref(i))
        return {f: getattr(i, f) for f, _ in L.SavedInfo._fields_}

    def __del__(self):
        try:
            if self.h:
                self.lib.gsr_saved_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Rasterizer:
    """A libgsr context: configuration, workspace and tuning cache."""

    def __init__(self, tile=(16, 16), batch: int = 256, sh_degree: int = 3, near: float = 0.2,
                 bg=(0.0, 0.0, 0.0), no_sync: bool = False, device=None):
        self.lib = L.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        cfg = L.Config()
        self.lib.gsr_config_default(C.byref(cfg))
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
        cfg.blend_batch = int(batch)
        cfg.sh_degree = int(sh_degree)
        cfg.near_plane = float(near)
        for i in range(3):
            cfg.bg[i] = float(bg[i])
        cfg.flags = L.GSR_FLAG_NO_SYNC if no_sync else 0
        self.cfg = cfg
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            code = self.lib.gsr_create(C.byref(h), C.byref(cfg))
        if code != 0:
            raise L.GsrError(code, "gsr_create failed")
        self.ctx = h

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.lib.gsr_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------------
    def _check(self, code):
        if code != 0:
            msg = self.lib.gsr_last_error(self.ctx)
            raise L.GsrError(code, msg.decode() if msg else "")

    def set_config(self, tile=None, batch=None, no_sync=None, profile=None, batch_bwd=None, pair_counts=None,
                   list_prefix=None):
        """list_prefix: >= 1 one list round; f in (0, 1) two rounds with the
        first over the nearest fraction f of the visible records; 0 two rounds
        with f chosen from the last synchronising forward's statistics."""
        if tile is not None:
            self.cfg.tile_w, self.cfg.tile_h = int(tile[0]), int(tile[1])
        if batch is not None:
            self.cfg.blend_batch = int(batch)
        if batch_bwd is not None:
            self.cfg.blend_batch_bwd = int(batch_bwd)
        if no_sync is not None:
            self.cfg.flags = (self.cfg.flags & ~L.GSR_FLAG_NO_SYNC) | (L.GSR_FLAG_NO_SYNC if no_sync else 0)
        if profile is not None:
            self.cfg.flags = (self.cfg.flags & ~L.GSR_FLAG_PROFILE) | (L.GSR_FLAG_PROFILE if profile else 0)
        if pair_counts is not None:
            self.cfg.flags = ((self.cfg.flags & ~L.GSR_FLAG_NO_PAIR_COUNTS) |
                              (0 if pair_counts else L.GSR_FLAG_NO_PAIR_COUNTS))
        if list_prefix is not None:
            self.cfg.list_prefix = float(list_prefix)
        self._check(self.lib.gsr_set_config(self.ctx, C.byref(self.cfg)))

    def stats(self) -> dict:
        """Kernel launches so far and per-phase device time of the profiled calls since the last read."""
        s = L.Stats()
        self._check(self.lib.gsr_get_stats(self.ctx, C.byref(s)))
        return dict(launches=int(s.launches),
                    phase_ms={p: float(s.phase_ms[i]) for i, p in enumerate(L.PHASES)},
                    calls={p: int(s.calls[i]) for i, p in enumerate(L.PHASES)})

    def get_config(self) -> dict:
        c = L.Config()
        self._check(self.lib.gsr_get_config(self.ctx, C.byref(c)))
        return dict(tile=(c.tile_w, c.tile_h), batch=c.blend_batch, sh_degree=c.sh_degree,
                    batch_bwd=c.blend_batch_bwd, list_prefix=c.list_prefix)

    def new_saved(self) -> _Saved:
        return _Saved(self)

    @staticmethod
    def _gaussians(means, log_scales, quats, opacity_logits, sh) -> L.Gaussians:
        for t in (means, log_scales, quats, opacity_logits, sh):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("Gaussian parameters must be contiguous float32 CUDA tensors")
        g = L.Gaussians()
        g.n = means.shape[0]
        g.means, g.log_scales, g.quats = means.data_ptr(), log_scales.data_ptr(), quats.data_ptr()
        g.opacity_logits, g.sh = opacity_logits.data_ptr(), sh.data_ptr()
        return g

    @staticmethod
    def _views(views: Sequence[CameraView]):
        arr = (L.View * len(views))()
        for i, v in enumerate(views):
            a = arr[i]
            a.width, a.height = int(v.width), int(v.height)
            a.fx, a.fy, a.cx, a.cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
            vm = np.ascontiguousarray(np.asarray(v.viewmat, np.float32).reshape(16))
            for k in range(16):
                a.viewmat[k] = float(vm[k])
            if v.subset is not None:
                if not (v.subset.is_cuda and v.subset.dtype in (torch.int32,) and v.subset.is_contiguous()):
                    raise ValueError("subset must be a contiguous int32 CUDA tensor")
                a.subset_count = int(v.subset.numel())
                a.subset = v.subset.data_ptr() if a.subset_count > 0 else _nonnull_ptr(v.subset.device)
            else:
                a.subset = None
                a.subset_count = 0
        return arr

    # -- raw calls -------------------------------------------------------------
    def forward(self, params, views: Sequence[CameraView], saved: Optional[_Saved] = None, out=None):
        """params: (means, log_scales, quats, opacity_logits, sh).  Returns (rgb, depth, alpha, saved)."""
        npix = sum(int(v.width) * int(v.height) for v in views)
        if out is None:
            dev = params[0].device
            out = (torch.empty(3 * npix, device=dev), torch.empty(npix, device=dev), torch.empty(npix, device=dev))
        rgb, depth, alpha = out
        saved = saved or self.new_saved()
        g = self._gaussians(*params)
        vs = self._views(views)
        o = L.Outputs(rgb.data_ptr(), depth.data_ptr(), alpha.data_ptr())
        self._check(self.lib.gsr_forward(self.ctx, C.byref(g), vs, len(views), C.byref(o), saved.h,
                                         _stream_ptr(rgb.device)))
        return rgb, depth, alpha, saved

    def backward(self, params, views, saved: _Saved, dl_rgb, dl_depth=None, dl_alpha=None, want_pose=True,
                 grads=None, want_focal=False):
        """Gradients (means, log_scales, quats, opacity_logits, sh, pose[V,6]
        or None, and with want_focal focal[V,2] = dL/d(fx, fy))."""
        means = params[0]
        if grads is None:
            grads = tuple(torch.empty_like(p) for p in params) + (
                torch.empty(len(views), 6, device=means.device) if want_pose else None,)
            if want_focal:
                grads = grads + (torch.empty(len(views), 2, device=means.device),)
        g = self._gaussians(*params)
        vs = self._views(views)
        gr = L.Grads(*(None if t is None else t.data_ptr() for t in grads))
        self._check(self.lib.gsr_backward(self.ctx, C.byref(g), vs, len(views), saved.h, _ptr(dl_rgb),
                                          _ptr(dl_depth), _ptr(dl_alpha), C.byref(gr), _stream_ptr(means.device)))
        return grads

    def check(self, saved: _Saved):
        self._check(self.lib.gsr_check(self.ctx, saved.h, _stream_ptr(self.device)))

    def insertion(self, gt: torch.Tensor, rendered: torch.Tensor, depth: torch.Tensor, views: Sequence[CameraView],
                  sigma: float = 1.0, tau_a: float = 0.2, index_cap: Optional[int] = None, out=None,
                  read_count: bool = True):
        """Insertion probability and scale initialisation (Sec. 3.2, Eq. 4-6)
        on the batch: gt, rendered [sum 3 W H] planar RGB per view, depth
        [sum W H].  Returns (p_a, scale, index of the inserted pixels, count);
        index holds the first index_cap (default: all pixels) ascending.
        read_count=False leaves everything on the device (no host wait):
        count is then the device tensor and index the whole buffer."""
        npix = sum(int(v.width) * int(v.height) for v in views)
        dev = gt.device
        cap = npix if index_cap is None else int(index_cap)
        p_a, scale, index = out if out is not None else (torch.empty(npix, device=dev), torch.empty(npix, device=dev),
                                                         torch.empty(max(cap, 1), dtype=torch.int32, device=dev))
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        prm = L.InsertParams(float(sigma), float(tau_a))
        vs = self._views(views)
        self._check(self.lib.gsr_insertion(self.ctx, C.byref(prm), vs, len(views), _ptr(gt), _ptr(rendered),
                                           _ptr(depth), _ptr(p_a), _ptr(scale), _ptr(index), cap, _ptr(count),
                                           _stream_ptr(dev)))
        if not read_count:
            return p_a, scale, index, count
        n = int(count.item())
        return p_a, scale, index[: min(n, cap)], n

    def rig_chain(self, pose_grads: torch.Tensor, keyframe_of_view, rel, n_keyframes: int, focal_grads=None,
                  camera_of_view=None, n_cameras: int = 0):
        """Rig parameter gradients (Sec. 3.1, 3.3) from the per-view ones:
        V_i = A_i V_m(k), rel [V, 3, 4] the A_i = [R_i | t_i] (host array),
        keyframe_of_view / camera_of_view [V] ints.  Returns a dict with
        "central" [K, 6] and, given camera_of_view, "camera_rel" [C, 6] and
        (with focal_grads) "camera_focal" [C, 2]; device tensors."""
        import numpy as np
        dev = pose_grads.device
        nv = int(pose_grads.shape[0])
        kf = np.ascontiguousarray(np.asarray(keyframe_of_view, np.int32).reshape(nv))
        A = np.ascontiguousarray(np.asarray(rel, np.float32).reshape(nv, 12))
        out = {"central": torch.empty(int(n_keyframes), 6, device=dev)}
        cam = None
        if camera_of_view is not None:
            cam = np.ascontiguousarray(np.asarray(camera_of_view, np.int32).reshape(nv))
            out["camera_rel"] = torch.empty(int(n_cameras), 6, device=dev)
            if focal_grads is not None:
                out["camera_focal"] = torch.empty(int(n_cameras), 2, device=dev)
        self._check(self.lib.gsr_rig_chain(
            self.ctx, nv, _ptr(pose_grads.contiguous()), _ptr(None if focal_grads is None else focal_grads.contiguous()),
            kf.ctypes.data, None if cam is None else cam.ctypes.data, A.ctypes.data, int(n_keyframes), int(n_cameras),
            _ptr(out["central"]), _ptr(out.get("camera_rel")), _ptr(out.get("camera_focal")), _stream_ptr(dev)))
        return out

    def merge(self, view: "CameraView", means: torch.Tensor, log_scales: torch.Tensor, sh: torch.Tensor,
              sample_pixels: torch.Tensor, scale_map: torch.Tensor, depth_map: torch.Tensor, gt: torch.Tensor,
              tau_d: float = 0.5, near_plane: float = 0.2) -> dict:
        """Inter-camera merging (Sec. 3.2, Eq. 7-8) of camera `view`'s samples
        (int32 pixel indices, e.g. from insertion()) with the existing
        Gaussians (means, log_scales [N, 3], sh [N, K, 3] or [N, 3]).  Returns
        device tensors: sample_action/means/scale/depth/dc and
        existing_action/dc (existing_dc holds the group's mean colour on the
        rows whose action is kept; the other rows are not written)."""
        dev = means.device
        n = int(means.shape[0])
        m = int(sample_pixels.numel())
        stride = int(sh.stride(0)) if n else 3
        out = {"sample_action": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
               "sample_means": torch.empty(max(m, 1), 3, device=dev),
               "sample_scale": torch.empty(max(m, 1), device=dev),
               "sample_depth": torch.empty(max(m, 1), device=dev),
               "sample_dc": torch.empty(max(m, 1), 3, device=dev),
               "existing_action": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
               "existing_dc": torch.empty(max(n, 1), 3, device=dev)}
        o = L.MergeOutputs(*(out[k].data_ptr() for k in ("sample_action", "sample_means", "sample_scale",
                                                         "sample_depth", "sample_dc", "existing_action",
                                                         "existing_dc")))
        prm = L.MergeParams(float(tau_d), float(near_plane))
        vs = self._views([view])
        self._check(self.lib.gsr_merge(self.ctx, C.byref(prm), vs, n, _ptr(means), _ptr(log_scales), _ptr(sh),
                                       stride, m, _ptr(sample_pixels), _ptr(scale_map), _ptr(depth_map), _ptr(gt),
                                       C.byref(o), _stream_ptr(dev)))
        for k in list(out):
            out[k] = out[k][: (m if k.startswith("sample") else n)]
        return out

    def dft_energy(self, images, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """X(I) of Eq. 10 for each image: images is a sequence of
        (tensor [3, H, W] or flat planar RGB, width, height, factor); factor n
        box-downsamples by n first (I^n).  Returns a device tensor [len]."""
        n = len(images)
        arr = (L.Image * max(n, 1))()
        dev = self.device
        for i, (t, w, h, f) in enumerate(images):
            if t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("images must be contiguous float32")
            dev = t.device
            arr[i] = L.Image(t.data_ptr(), int(w), int(h), int(f))
        x = out if out is not None else torch.empty(n, device=dev)
        self._check(self.lib.gsr_dft_energy(self.ctx, arr, n, _ptr(x), _stream_ptr(dev)))
        return x

    def frequency_schedule(self, x_gt: torch.Tensor, x_rendered: torch.Tensor, x_gt_level=None, tau_f: float = 2.0,
                           uniforms: Optional[torch.Tensor] = None) -> dict:
        """Eq. 9 and 12 with the scheduler's decisions: r, r_level, level_up
        (r_level < tau_f) per frame and one frame index per uniform, drawn
        with probability proportional to r."""
        dev = x_gt.device
        n = int(x_gt.numel())
        out = {"r": torch.empty(n, device=dev)}
        if x_gt_level is not None:
            out["r_level"] = torch.empty(n, device=dev)
            out["level_up"] = torch.empty(n, dtype=torch.int32, device=dev)
        ns = 0 if uniforms is None else int(uniforms.numel())
        if uniforms is not None:
            out["samples"] = torch.empty(max(ns, 1), dtype=torch.int32, device=dev)
        self._check(self.lib.gsr_frequency_schedule(
            self.ctx, n, _ptr(x_gt), _ptr(x_gt_level), _ptr(x_rendered), float(tau_f), _ptr(uniforms), ns,
            _ptr(out["r"]), _ptr(out.get("r_level")), _ptr(out.get("level_up")), _ptr(out.get("samples")),
            _stream_ptr(dev)))
        if "samples" in out:
            out["samples"] = out["samples"][:ns]
        return out

    def tune(self, params, views, dl_rgb, saved=None, out=None, grads=None) -> dict:
        npix = sum(int(v.width) * int(v.height) for v in views)
        dev = params[0].device
        out = out or (torch.empty(3 * npix, device=dev), torch.empty(npix, device=dev), torch.empty(npix, device=dev))
        grads = grads or tuple(torch.empty_like(p) for p in params) + (torch.empty(len(views), 6, device=dev),)
        saved = saved or self.new_saved()
        g = self._gaussians(*params)
        vs = self._views(views)
        o = L.Outputs(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        gr = L.Grads(*(t.data_ptr() for t in grads))
        best = L.Config()
        self._check(self.lib.gsr_tune(self.ctx, C.byref(g), vs, len(views), C.byref(o), saved.h, _ptr(dl_rgb),
                                      C.byref(gr), C.byref(best), _stream_ptr(dev)))
        self.cfg = best
        return dict(tile=(best.tile_w, best.tile_h), batch=best.blend_batch, batch_bwd=best.blend_batch_bwd)

    # -- parity exports --------------------------------------------------------
    def debug_lists(self, saved: _Saved):
        info = saved.info()
        dev = self.device
        # list positions: both regions' after a two-round forward
        m, nt = info["list_span"], info["n_tiles"]
        keys = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
        vals = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        ranges = torch.empty(max(nt, 1), 2, dtype=torch.int32, device=dev)
        self._check(self.lib.gsr_debug_lists(saved.h, _ptr(keys), _ptr(vals), _ptr(ranges), _stream_ptr(dev)))
        return keys[:m], vals[:m], ranges[:nt]

    def debug_list_slice(self, saved: _Saved, first: int, count: int):
        """(keys, vals) of sorted-list positions [first, first + count)."""
        dev = self.device
        keys = torch.empty(max(count, 1), dtype=torch.int64, device=dev)
        vals = torch.empty(max(count, 1), dtype=torch.int32, device=dev)
        self._check(self.lib.gsr_debug_list_slice(saved.h, int(first), int(count), _ptr(keys), _ptr(vals),
                                                  _stream_ptr(dev)))
        return keys[:count], vals[:count]

    def debug_ranges(self, saved: _Saved):
        nt = saved.info()["n_tiles"]
        ranges = torch.empty(max(nt, 1), 2, dtype=torch.int32, device=self.device)
        self._check(self.lib.gsr_debug_lists(saved.h, None, None, _ptr(ranges), _stream_ptr(self.device)))
        return ranges[:nt]

    def debug_records(self, saved: _Saved):
        info = saved.info()
        n = info["n_records"]
        dev = self.device
        rec = torch.empty(max(n, 1), 16, device=dev)
        rect = torch.empty(max(n, 1), 4, dtype=torch.int32, device=dev)
        flags = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self._check(self.lib.gsr_debug_records(saved.h, _ptr(rec), _ptr(rect), _ptr(flags), _stream_ptr(dev)))
        return rec[:n], rect[:n], flags[:n]

    def debug_pixels(self, saved: _Saved):
        n = saved.info()["n_pixels"]
        tf = torch.empty(n, device=self.device)
        nc = torch.empty(n, dtype=torch.int32, device=self.device)
        self._check(self.lib.gsr_debug_pixels(saved.h, _ptr(tf), _ptr(nc), _stream_ptr(self.device)))
        return tf, nc

    def debug_set_wait(self, wait_ns: int = 0, withhold_prefix: bool = False):
        """Limit of every device wait of later calls (0: the default 2 s);
        withhold_prefix makes the forward's first scan block keep its prefix,
        so the later blocks' waits run out (tests of the timeout path)."""
        self._check(self.lib.gsr_debug_set_wait(self.ctx, int(wait_ns),
                                                L.GSR_DEBUG_WITHHOLD_PREFIX if withhold_prefix else 0))

    def debug_record_grads(self, saved: _Saved):
        n = saved.info()["n_records"]
        g = torch.empty(max(n, 1), 12, device=self.device)
        self._check(self.lib.gsr_debug_record_grads(saved.h, _ptr(g), _stream_ptr(self.device)))
        return g[:n]


def l1_loss_grad(rgb: torch.Tensor, target: torch.Tensor, dl: Optional[torch.Tensor] = None,
                 loss: Optional[torch.Tensor] = None):
    """L1 loss mean|rgb - target| and its gradient, computed by libgsr."""
    lib = L.load()
    dl = torch.empty_like(rgb) if dl is None else dl
    code = lib.gsr_l1_loss_grad(_ptr(rgb), _ptr(target), rgb.numel(), _ptr(dl), _ptr(loss), _stream_ptr(rgb.device))
    if code != 0:
        raise L.GsrError(code, "gsr_l1_loss_grad failed")
    return dl, loss


def _require_zero(name: str, t: Optional[torch.Tensor], shape) -> None:
    """The pose and focal inputs are perturbations at which the gradient is
    taken (the renderer uses the views' own matrices and intrinsics): they
    must be zeros of the given shape.  Reads them back to the host."""
    if t is None:
        return
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if bool((t.detach() != 0).any()):
        raise ValueError(f"{name} must be zero: its gradient is taken at zero; fold a non-zero update into "
                         "the views (viewmat / fx, fy) instead")


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, pose_delta, focal_delta, raster, views):
        _require_zero("pose_delta", pose_delta, (len(views), 6))
        _require_zero("focal_delta", focal_delta, (len(views), 2))
        params = (means.detach().contiguous(), log_scales.detach().contiguous(), quats.detach().contiguous(),
                  opacity_logits.detach().contiguous(), sh.detach().contiguous())
        rgb, depth, alpha, saved = raster.forward(params, views)
        ctx.raster, ctx.views, ctx.saved, ctx.params = raster, views, saved, params
        ctx.want_pose = pose_delta is not None
        ctx.want_focal = focal_delta is not None
        ctx.rgb_numel = rgb.numel()
        return rgb, depth, alpha

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_alpha):
        # the library needs an rgb gradient; a loss on depth or alpha alone gives none
        d_rgb = d_rgb.contiguous() if d_rgb is not None else \
            torch.zeros(ctx.rgb_numel, device=ctx.params[0].device, dtype=torch.float32)
        grads = ctx.raster.backward(ctx.params, ctx.views, ctx.saved, d_rgb,
                                    None if d_depth is None else d_depth.contiguous(),
                                    None if d_alpha is None else d_alpha.contiguous(), want_pose=ctx.want_pose,
                                    want_focal=ctx.want_focal)
        gm, gls, gq, go, gsh, gpose = grads[:6]
        gfocal = grads[6] if ctx.want_focal else None
        return gm, gls, gq, go, gsh, gpose, gfocal, None, None


def rasterize(means, log_scales, quats, opacity_logits, sh, views: Sequence[CameraView],
              raster: Rasterizer, pose_delta: Optional[torch.Tensor] = None,
              focal_delta: Optional[torch.Tensor] = None):
    """Differentiable render of all ``views`` in one batched call.

    Returns flat (rgb [3 sum HW], depth [sum HW], alpha [sum HW]); use
    ``split_images`` for per-view views.  ``pose_delta`` ([V, 6]) and
    ``focal_delta`` ([V, 2]) must be zeros: they are inputs whose gradients are
    dL/d(rho, omega) of each view's left-perturbed pose and dL/d(fx, fy); a
    non-zero value raises ValueError (the views carry the pose and focal).
    """
    return _RasterizeFn.apply(means, log_scales, quats, opacity_logits, sh, pose_delta, focal_delta, raster,
                              list(views))
