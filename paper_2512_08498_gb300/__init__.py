"""GB300-native differentiable tile-based Gaussian-splatting rasterizer.

The renderer of the per-keyframe optimisation in "On-the-fly Large-scale 3D
Reconstruction from Multi-Camera Rigs" (Sec. 3.3): forward and backward,
including se(3) camera-pose gradients, batched over all rig cameras and
keyframes of a local window.  All work runs in hand-written sm_103a CUDA
kernels behind the C ABI of ``include/gsr.h`` (``libgsr.so``, built in-tree
by ``build.py``); this package only marshals arguments.

Import is cheap and GPU-free: ``scenes`` (seeded synthetic inputs) works on
any machine; ``Rasterizer`` / ``rasterize`` load libgsr.so on first use and
raise if it is missing.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "Rasterizer", "rasterize", "CameraView", "to_camera_views", "split_images",
           "l1_loss_grad", "build"]


def __getattr__(name):
    if name in ("Rasterizer", "rasterize", "CameraView", "to_camera_views", "split_images", "l1_loss_grad",
                "pixel_offsets"):
        from . import rasterizer
        return getattr(rasterizer, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
