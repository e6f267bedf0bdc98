"""The allocation-free forward render, gsr_forward_noalloc, against gsr_forward.

Some callers cannot allocate device memory while they render: a process that
reserved its whole device budget when it started, or code running where
cudaMalloc is not permitted.  For them libgsr has one forward whose workspace
is a fixed array compiled into the library.  These tests call it through the
C ABI, twice in a row (the second call reuses the array the first one left
behind), and compare its images with those of the ordinary forward on the same
inputs; they also check that a batch beyond its limits is refused before any
device work.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2512_08498_gb300 import _lib as L  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views  # noqa: E402

import _parity as P  # noqa: E402


def _scene():
    rng = np.random.default_rng(12)
    n = 3000
    views = [scenes.pinhole(70, 45, f=60.0),
             scenes.pinhole(48, 40, f=50.0, viewmat=scenes.look_from([0.1, -0.05, -0.3], yaw_deg=8.0)),
             scenes.pinhole(64, 36, f=44.0, viewmat=scenes.look_from([0.0, 0.05, -0.1], roll_deg=20.0),
                            subset=np.sort(rng.choice(n, n // 3, replace=False)).astype(np.uint32))]
    return scenes.random_scene(12, n, views, 3, bg=(0.1, 0.2, 0.3))


def _call_noalloc(raster, params, cams, npix):
    lib = L.load()
    dev = params[0].device
    rgb = torch.full((3 * npix,), -1.0, device=dev)
    depth = torch.full((npix,), -1.0, device=dev)
    alpha = torch.full((npix,), -1.0, device=dev)
    g = Rasterizer._gaussians(*params)
    vs = Rasterizer._views(cams)
    out = L.Outputs(rgb.data_ptr(), depth.data_ptr(), alpha.data_ptr())
    code = lib.gsr_forward_noalloc(C.byref(raster.cfg), C.byref(g), vs, len(cams), C.byref(out),
                                   C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    torch.cuda.synchronize(dev)
    return code, rgb, depth, alpha


def test_noalloc_forward_matches_forward_on_two_calls():
    sc = _scene()
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    npix = sum(v.width * v.height for v in sc.views)
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    rgb, depth, alpha, _ = r.forward(params, cams)
    ref = [t.cpu().numpy() for t in (rgb, depth, alpha)]
    for _ in range(2):
        code, rgb2, depth2, alpha2 = _call_noalloc(r, params, cams, npix)
        assert code == L.GSR_OK
        got = [t.cpu().numpy() for t in (rgb2, depth2, alpha2)]
        assert np.abs(got[0] - ref[0]).max() <= P.IMG_TOL
        assert np.abs(got[2] - ref[2]).max() <= P.IMG_TOL
        assert (np.abs(got[1] - ref[1]) / np.maximum(1.0, np.abs(ref[1]))).max() <= P.IMG_TOL


def test_noalloc_refuses_batches_beyond_its_limits():
    sc = _scene()
    sc.views = [scenes.pinhole(1024, 1024, f=900.0)]   # 1,048,576 pixels > GSR_NOALLOC_MAX_PIXELS
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    code, rgb, _, _ = _call_noalloc(r, params, cams, 1024 * 1024)
    assert code == L.GSR_ERR_NOT_SUPPORTED
    assert bool((rgb == -1.0).all())      # nothing was written
