"""GPU parity of the camera gradients beyond the per-view pose: the focal
lengths (dL/dfx, dL/dfy per view, Sec. 3.1) and the rig chain (Sec. 3.1, 3.3)
that turns per-view pose and focal gradients into per-keyframe central-pose,
per-camera relative-transform and per-camera focal gradients."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_08498_gb300 import scenes  # noqa: E402
from paper_2512_08498_gb300._lib import GsrError  # noqa: E402
from paper_2512_08498_gb300.scenes import pinhole, look_from  # noqa: E402

import _parity as P  # noqa: E402


def _rig(seed=31, n=900):
    """Three keyframes of a three-camera rig, V_i = A_c V_m(k); ragged sizes."""
    central = [look_from([0.0, 0.0, 0.0]), look_from([0.2, -0.05, 0.3], yaw_deg=6.0, pitch_deg=-3.0),
               look_from([0.35, 0.02, 0.6], yaw_deg=11.0)]
    A = [np.eye(4), look_from([0.12, 0.02, 0.05], yaw_deg=-9.0, roll_deg=2.0),
         look_from([-0.15, 0.0, 0.04], yaw_deg=14.0, pitch_deg=1.5)]
    sizes = [(70, 45, 60.0), (48, 40, 50.0), (33, 31, 40.0)]
    views, kf, cam, rel = [], [], [], []
    for k, Vm in enumerate(central):
        for c, Ac in enumerate(A):
            w, h, f = sizes[c]
            A32 = np.asarray(Ac, np.float32).astype(np.float64)
            views.append(pinhole(w, h, f=f, viewmat=A32 @ np.asarray(Vm, np.float64)))
            kf.append(k); cam.append(c); rel.append(A32[:3, :])
    sc = scenes.random_scene(seed, n, views, 3, bg=(0.1, 0.2, 0.3))
    return sc, kf, cam, np.stack(rel)


def test_focal_gradients_per_view():
    sc, _, _, _ = _rig()
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref, seed=3)
    g = P.run_gpu(sc, grads=up_g)
    go = o.backward(up_o[0], up_o[1], up_o[2])
    errs = P.compare_grads(g, go)
    assert np.abs(go["focal"]).max() > 0 and errs["focal"] <= P.GRAD_TOL


def test_rig_chain_against_the_oracle():
    sc, kf, cam, rel = _rig()
    o = oracle.Oracle(sc)
    ref = o.forward()
    up_o, up_g = P.upstream(sc, o, ref, seed=4)
    g = P.run_gpu(sc, grads=up_g)
    go = o.backward(up_o[0], up_o[1], up_o[2])
    r = g["raster"]
    dev = P.device()
    pose = torch.from_numpy(g["grads"]["pose"].astype(np.float32)).to(dev)
    focal = torch.from_numpy(g["grads"]["focal"].astype(np.float32)).to(dev)
    out = r.rig_chain(pose, kf, rel, 3, focal_grads=focal, camera_of_view=cam, n_cameras=3)
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    # (1) the whole chain against the oracle's per-view gradients: the gradient bar
    exp = oracle.rig_chain(go["pose"], kf, rel, 3, focal_grads=go["focal"], camera_of_view=cam, n_cameras=3)
    for k in ("central", "camera_rel", "camera_focal"):
        assert P.rel_l2(got[k], exp[k]) <= P.GRAD_TOL, k
    # (2) the chain alone, on the same binary32 per-view inputs: binary64 sums
    # rounded once, so within a few binary32 ulps of the oracle's
    exp32 = oracle.rig_chain(g["grads"]["pose"], kf, rel, 3, focal_grads=g["grads"]["focal"],
                             camera_of_view=cam, n_cameras=3)
    for k in ("central", "camera_rel", "camera_focal"):
        scale = np.abs(exp32[k]).max()
        assert np.abs(got[k] - exp32[k]).max() <= 4e-7 * scale, k


def test_rig_chain_without_camera_outputs_and_bad_indices():
    sc, kf, cam, rel = _rig()
    dev = P.device()
    from paper_2512_08498_gb300.rasterizer import Rasterizer
    r = Rasterizer(device=dev)
    rng = np.random.default_rng(5)
    pose = rng.normal(size=(len(kf), 6)).astype(np.float32)
    out = r.rig_chain(torch.from_numpy(pose).to(dev), kf, rel, 3)
    assert set(out) == {"central"}
    exp = oracle.rig_chain(pose, kf, rel, 3)
    c = out["central"].cpu().numpy()
    assert np.abs(c - exp["central"]).max() <= 4e-7 * np.abs(exp["central"]).max()
    bad = list(kf)
    bad[2] = 3
    with pytest.raises(GsrError):
        r.rig_chain(torch.from_numpy(pose).to(dev), bad, rel, 3)
    with pytest.raises(GsrError):
        r.rig_chain(torch.from_numpy(pose).to(dev), kf, rel, 3, camera_of_view=[0] * (len(kf) - 1) + [7],
                    n_cameras=3)
