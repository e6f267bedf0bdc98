"""The timeout path of the bounded device waits, exercised without a fault.

Every device-side wait of libgsr (mbarrier waits on bulk copies, decoupled
look-back spins) gives up after a limit, sets the timeout bit of the call's
status word and lets its kernel finish; every later kernel of the call skips
its work, and the call reports GSR_ERR_TIMEOUT.  Here the limit is cut to
200 microseconds and the first block of the preprocess's single-pass scan
withholds its prefix (a flag nothing else sets), so every later block's wait
runs out.  The call must report the timeout, synchronously and through
gsr_check after an unsynchronised forward + backward, and the next ordinary
call on the same context must match the oracle as everywhere else.
"""
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
from paper_2512_08498_gb300.scenes import look_from, pinhole  # noqa: E402

import _parity as P  # noqa: E402


def _scene():
    # 2 x 3000 records: several look-back tickets of the preprocess scan
    views = [pinhole(70, 45, f=60.0),
             pinhole(48, 40, f=50.0, viewmat=look_from([0.1, -0.05, -0.3], yaw_deg=8.0))]
    return scenes.random_scene(90, 3000, views, 2, bg=(0.1, 0.2, 0.3))


def test_withheld_prefix_times_out_then_the_context_recovers():
    sc = _scene()
    dev = P.device()
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg, device=dev)
    params = P.params_of(sc, dev)
    cams = to_camera_views(sc.views, dev)

    r.debug_set_wait(wait_ns=200_000, withhold_prefix=True)
    with pytest.raises(L.GsrError) as e:
        r.forward(params, cams)
    assert e.value.code == L.GSR_ERR_TIMEOUT

    # unsynchronised: forward and backward return at once, gsr_check reports
    r.set_config(no_sync=True)
    rgb, depth, alpha, saved = r.forward(params, cams)
    r.backward(params, cams, saved, torch.zeros_like(rgb))
    with pytest.raises(L.GsrError) as e:
        r.check(saved)
    assert e.value.code == L.GSR_ERR_TIMEOUT

    # back to the default limit, no withholding: parity on the same context
    r.set_config(no_sync=False)
    r.debug_set_wait(0, False)
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref)
    g = P.run_gpu(sc, grads=up_g, raster=r)
    P.compare_records(g, o)
    P.compare_lists(g, o)
    P.compare_pixels(g, o, ref)
    P.compare_counters(g, o, ref, with_bwd=True)
    P.compare_images(g, ref)
    P.compare_grads(g, o.backward(*up_o))


def test_unknown_debug_flags_are_refused():
    r = Rasterizer(tile=(16, 16), batch=256, sh_degree=0)
    assert r.lib.gsr_debug_set_wait(r.ctx, 0, 2) == L.GSR_ERR_INVALID_ARG
