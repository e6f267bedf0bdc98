"""View sharding of one batch on one GPU (the multi-GPU split, run serially).

A batch sharded over ranks renders each rank's block of views against the
same Gaussians and sums the ranks' parameter gradients with one all-reduce.
Here the two blocks of a world-size-2 split run one after the other on one
GPU, each into its own flat gradient buffer (paper_2512_08498_gb300.sharding),
and the buffers are added on the device -- what the all-reduce computes.
The sum must equal the gradients of the whole batch rendered in one call and
the oracle's within 1e-4 relative L2, and each block's pose gradients the
corresponding rows.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300.rasterizer import Rasterizer, pixel_offsets, to_camera_views  # noqa: E402
from paper_2512_08498_gb300.scenes import look_from, pinhole  # noqa: E402
from paper_2512_08498_gb300.sharding import GradBuffer, shard_views  # noqa: E402

import _parity as P  # noqa: E402


def _batch():
    n = 2000
    rng = np.random.default_rng(21)
    views = [pinhole(70, 45, f=60.0),
             pinhole(48, 40, f=50.0, viewmat=look_from([0.1, -0.05, -0.3], yaw_deg=8.0, pitch_deg=-4.0)),
             pinhole(33, 31, f=40.0, viewmat=look_from([-0.2, 0.1, 0.2], yaw_deg=-10.0),
                     subset=np.sort(rng.choice(n, n // 2, replace=False)).astype(np.uint32)),
             pinhole(64, 36, f=44.0, viewmat=look_from([0.0, 0.05, -0.1], roll_deg=20.0))]
    return scenes.random_scene(21, n, views, 3, bg=(0.1, 0.2, 0.3))


def _render(r, params, cams, ups, buf):
    npix = sum(c.width * c.height for c in cams)
    rgb, depth, alpha = (torch.empty(3 * npix, device=P.device()), torch.empty(npix, device=P.device()),
                         torch.empty(npix, device=P.device()))
    _, _, _, saved = r.forward(params, cams, out=(rgb, depth, alpha))
    pose = torch.empty(len(cams), 6, device=P.device())
    r.backward(params, cams, saved, *ups, grads=buf.tensors() + (pose,))
    return pose


def test_two_view_shards_sum_to_the_whole_batch():
    sc = _batch()
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref)
    dev = P.device()
    params = P.params_of(sc, dev)
    cams = to_camera_views(sc.views, dev)
    offs = pixel_offsets(cams)
    ups = [torch.from_numpy(x).to(dev) for x in up_g]
    r = Rasterizer(tile=sc.tile, batch=256, sh_degree=sc.sh_degree, bg=sc.bg, device=dev)

    whole = GradBuffer(sc.n, sc.sh_degree, dev)
    pose_whole = _render(r, params, cams, ups, whole)

    total = torch.zeros_like(whole.flat)
    poses = []
    for rank in range(2):
        a, b = shard_views(cams, rank, 2)
        assert b > a
        pa, pb = offs[a], offs[b]
        part = (ups[0][3 * pa:3 * pb], ups[1][pa:pb], ups[2][pa:pb])
        buf = GradBuffer(sc.n, sc.sh_degree, dev)
        poses.append((a, b, _render(r, params, cams[a:b], part, buf)))
        total += buf.flat          # the all-reduce's sum
    assert P.rel_l2(total.cpu().numpy(), whole.flat.cpu().numpy()) <= 1e-5
    go = o.backward(*up_o)
    summed = GradBuffer(sc.n, sc.sh_degree, "cpu")
    summed.flat.copy_(total.cpu())
    for name, t in zip(P.PARAM_NAMES, summed.tensors()):
        assert P.rel_l2(t.numpy(), go[name]) <= P.GRAD_TOL, name
    for a, b, p in poses:
        assert P.rel_l2(p.cpu().numpy(), pose_whole[a:b].cpu().numpy()) <= 1e-5
        assert P.rel_l2(p.cpu().numpy(), go["pose"][a:b]) <= P.GRAD_TOL


def test_grad_buffer_layout():
    buf = GradBuffer(5, 3, P.device())
    m, l, q, o, s = buf.tensors()
    assert q.data_ptr() % 16 == 0 and q.shape == (5, 4)
    assert m.shape == (5, 3) and l.shape == (5, 3) and o.shape == (5,) and s.shape == (5, 16, 3)
    assert buf.bytes_per_gaussian() == 4 * (4 + 3 + 3 + 1 + 48) == 236
