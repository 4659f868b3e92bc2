"""Non-finite inputs are reported, not rendered silently and not faulted.

Fitting by gradient descent (Sec. 3.1) is where NaN or infinite parameters
arise. The forward preprocess reads every parameter once and latches a status
bit when one is not finite; a synchronising render returns
DDGS_ERR_NONFINITE (its outputs are still written), a no-sync render leaves
it to ddgs_sync_status. The faults are made on the host: values written into
the input arrays before the call.
"""
import numpy as np
import pytest
import torch

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

DDGS_ERR_NONFINITE = 3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2406_02518_gb300 import build
    build.build()
    B.load()
    assert B.device_supported(), "needs an sm_103 (GB300) device"


def _inputs():
    scene = syn.uniform_cloud(800, seed=31)
    poses = np.stack([syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])),
                      syn.pose_matrix(syn.rot_y(0.4), np.array([0.0, 0.1, 2.2]))]).astype(np.float32)
    views = syn.Views(poses, syn.detector(2, 4.0, 8.0 / 48), 48, 48)
    return scene, views, syn.Settings(near_plane=0.2)


def _poison(cloud, gv, where, value):
    """Write one non-finite value into the named input (host-side fault)."""
    if where == "logit":
        cloud.opacity_logits[17] = value
    elif where == "feat_iso":
        cloud.feat_iso[3, 5] = value
    elif where == "feat_dir":
        cloud.feat_dir[2, 1] = value
    elif where == "log_scale":
        cloud.log_scales[40, 2] = value
    elif where == "mean":
        cloud.means[9, 0] = value
    elif where == "quat":
        cloud.quats[100, 3] = value
    elif where == "b_iso":
        cloud.b_iso[4] = value
    elif where == "B_dir":
        cloud.B_dir[1, 6] = value
    elif where == "pose":
        gv.world_to_cam[1, 2, 3] = value
    else:
        raise ValueError(where)


PLACES = ["logit", "feat_iso", "feat_dir", "log_scale", "mean", "quat", "b_iso", "B_dir", "pose"]


@pytest.mark.parametrize("value", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("where", PLACES)
def test_synchronising_render_reports_nonfinite(where, value):
    scene, views, st = _inputs()
    cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
    cfg = B.config_from_settings(st)
    ws = B.Workspace()
    try:
        clean, _, _ = B.render(cloud, gv, cfg, ws)
        clean = clean.clone()
        _poison(cloud, gv, where, value)
        with pytest.raises(B.DDGSError) as e:
            B.render(cloud, gv, cfg, ws)
        assert e.value.code == DDGS_ERR_NONFINITE
        torch.cuda.synchronize()  # the context is intact
        assert ws.sync_status() == 0  # reported once, then cleared
        # a finite cloud renders again, bit for bit as before
        cloud2, gv2 = B.cloud_from_arrays(scene), B.views_from_arrays(views)
        img, _, _ = B.render(cloud2, gv2, cfg, ws)
        torch.cuda.synchronize()
        assert torch.equal(img, clean)
    finally:
        ws.close()


@pytest.mark.parametrize("where", ["logit", "feat_dir", "pose"])
def test_no_sync_render_latches_nonfinite(where):
    scene, views, st = _inputs()
    cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
    ws = B.Workspace()
    try:
        B.render(cloud, gv, B.config_from_settings(st), ws)
        torch.cuda.synchronize()
        ws.reserve(views.n_views * scene.n, 2 * ws.pairs() + 4096, 2 * 9)
        cfg = B.config_from_settings(st, no_sync=True)
        _poison(cloud, gv, where, float("nan"))
        img, tf, nl = B.render(cloud, gv, cfg, ws)
        g = B.render_backward(cloud, gv, cfg, ws, torch.ones_like(img), tf, nl, want=["means"])
        torch.cuda.synchronize()
        assert ws.sync_status() == DDGS_ERR_NONFINITE
        assert ws.sync_status() == 0
        assert g["means"].shape == cloud.means.shape
    finally:
        ws.close()


def test_finite_inputs_report_nothing():
    scene, views, st = _inputs()
    cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
    ws = B.Workspace()
    try:
        for cfg in (B.config_from_settings(st), B.config_from_settings(st, batch_depth=32)):
            B.render(cloud, gv, cfg, ws)
        assert ws.sync_status() == 0
    finally:
        ws.close()
