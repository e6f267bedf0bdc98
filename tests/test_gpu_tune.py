"""The autotuner (gsr_tune): it picks a supported tile shape, blend batch and
backward batch, caches the choice per batch signature, and the configuration
it leaves in the context renders and differentiates exactly as the oracle
does for that tile shape."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.scenes import pinhole, look_from  # noqa: E402

import _parity as P  # noqa: E402


def test_tune_then_parity():
    from paper_2512_08498_gb300.rasterizer import Rasterizer, to_camera_views
    views = [pinhole(96, 64, f=70.0), pinhole(80, 72, f=60.0, viewmat=look_from([0.1, 0.0, -0.2], yaw_deg=6.0))]
    sc = scenes.random_scene(21, 3000, views, 3, bg=(0.1, 0.2, 0.3))
    dev = P.device()
    r = Rasterizer(sh_degree=3, bg=sc.bg, device=dev)
    params = P.params_of(sc, dev)
    cams = to_camera_views(sc.views, dev)
    npix = sum(v.width * v.height for v in sc.views)
    dl = torch.from_numpy(np.random.default_rng(1).standard_normal(3 * npix).astype(np.float32)).to(dev)
    best = r.tune(params, cams, dl)
    assert tuple(best["tile"]) in {(16, 16), (32, 8), (8, 32)}
    assert best["batch"] in (128, 256, 512) and best["batch_bwd"] in (0, 128, 256, 512)
    assert r.tune(params, cams, dl) == best   # cached for this batch signature
    # the tuned configuration against the oracle for its tile shape
    tile = tuple(best["tile"])
    sc.tile = tile
    o = oracle.Oracle(sc, tile=tile)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref, seed=2)
    g = P.run_gpu(sc, tile=tile, grads=up_g, raster=r)
    P.compare_lists(g, o)
    P.compare_pixels(g, o, ref)
    P.compare_images(g, ref)
    go = o.backward(up_o[0], up_o[1], up_o[2], want_grec=True)
    P.compare_grads(g, go)
    P.compare_record_grads(g, go)
