"""The allocation-free forward render, gsr_forward_noalloc, against gsr_forward.

Some callers cannot allocate device memory while they render: a process that
reserved its whole device budget when it started, or code running where
cudaMalloc is not permitted.  For them libgsr has one forward whose workspace
is a fixed array compiled into the library.  These tests call it through the
C ABI, twice in a row (the second call reuses the array the first one left
behind), and compare its images with those of the ordinary forward on the same
inputs (bit for bit: the same kernels run in the same configuration) and with
the CPU oracle's (within the image tolerance).  They also check that a batch
beyond its size limits is refused before any device work, and that a batch
whose tile instances overflow the fixed array is reported as such and leaves
the next call correct.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
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


def _images(ts):
    return [t.cpu().numpy() for t in ts]


def test_noalloc_forward_matches_forward_on_two_calls():
    sc = _scene()
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    npix = sum(v.width * v.height for v in sc.views)
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    rgb, depth, alpha, _ = r.forward(params, cams)
    ref = _images((rgb, depth, alpha))
    o = oracle.Oracle(sc)
    oref = o.forward()
    for _ in range(2):
        code, rgb2, depth2, alpha2 = _call_noalloc(r, params, cams, npix)
        assert code == L.GSR_OK
        got = _images((rgb2, depth2, alpha2))
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        P.compare_images({"rgb": got[0], "depth": got[1], "alpha": got[2]}, oref)


def _overflow_scene():
    """60,000 large opaque Gaussians on one 704x704 view: within the record,
    pixel and tile limits, but each keeps about 20 of its tiles after
    culling, far more than GSR_NOALLOC_MAX_INSTANCES in total."""
    rng = np.random.default_rng(5)
    n, W, f = 60000, 704, 600.0
    z = rng.uniform(3.0, 6.0, n)
    u, v = rng.uniform(0, W, n), rng.uniform(0, W, n)
    means = np.stack([(u - W / 2) * z / f, (v - W / 2) * z / f, z], 1).astype(np.float32)
    log_scales = np.log(np.repeat((13.0 * z / f)[:, None], 3, 1)).astype(np.float32)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    sh = rng.uniform(-0.5, 0.5, (n, 1, 3)).astype(np.float32)
    return scenes.Scene("overflow", means, log_scales, quats, np.full(n, 2.0, np.float32), sh, 0,
                        [scenes.pinhole(W, W, f=f)])


def test_noalloc_reports_instance_overflow_then_recovers():
    big = _overflow_scene()
    r = Rasterizer(tile=big.tile, batch=256, sh_degree=0, bg=big.bg)
    params = P.params_of(big)
    cams = to_camera_views(big.views)
    _, _, _, saved = r.forward(params, cams)
    assert saved.info()["n_instances"] > L.GSR_NOALLOC_MAX_INSTANCES
    code, _, _, _ = _call_noalloc(r, params, cams, 704 * 704)
    assert code == L.GSR_ERR_CAPACITY
    # the next call on the shared array starts clean
    sc = _scene()
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    npix = sum(v.width * v.height for v in sc.views)
    r2 = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    ref = _images(r2.forward(params, cams)[:3])
    code, rgb, depth, alpha = _call_noalloc(r2, params, cams, npix)
    assert code == L.GSR_OK
    for a, b in zip(_images((rgb, depth, alpha)), ref):
        assert np.array_equal(a, b)


def test_noalloc_refuses_batches_beyond_its_limits():
    sc = _scene()
    sc.views = [scenes.pinhole(1024, 1024, f=900.0)]   # 1,048,576 pixels > GSR_NOALLOC_MAX_PIXELS
    params = P.params_of(sc)
    cams = to_camera_views(sc.views)
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg)
    code, rgb, _, _ = _call_noalloc(r, params, cams, 1024 * 1024)
    assert code == L.GSR_ERR_NOT_SUPPORTED
    assert bool((rgb == -1.0).all())      # nothing was written
