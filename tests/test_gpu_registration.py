"""GPU: pose registration through the renderer (Sec. 4.3): Adam (lr 0.05) on a
6-DoF correction from the isocenter pose, several candidates batched in one
render per iteration, targets rendered at known poses of a phantom cloud."""
import numpy as np
import pytest
import torch

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import registration as reg
from paper_2406_02518_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_batched_registration_converges_on_phantom():
    ph = syn.make_phantom(128, seed=3)
    scene = syn.gaussians_from_phantom(ph, 60_000, seed=3)
    st = syn.Settings(near_plane=0.1 * syn.SID_MM)
    cfg = B.config_from_settings(st)
    cloud = B.cloud_from_arrays(scene)
    H = W = 128
    V = 4
    base = syn.ap_pose(syn.SID_MM)[0].astype(np.float64)
    rng = np.random.default_rng(11)
    true = reg.perturbed_poses(rng, base, V, max_deg=4.0, max_mm=6.0)
    det = torch.as_tensor(syn.detector(V, syn.SDD_MM, 256.0 / W), device="cuda")
    ws = B.Workspace()
    targets, _, _ = B.render(cloud, B.Views(torch.as_tensor(true, device="cuda"), det, H, W), cfg, ws)
    targets = targets.clone()
    init = torch.as_tensor(base, device="cuda")
    rot0 = reg.rotation_error_deg(np.repeat(base[None, :, :3], V, 0), true[:, :, :3])
    tr0 = reg.translation_error_mm(np.repeat(base[None], V, 0), true)
    res = reg.register(cloud, det, H, W, targets, init, cfg, iters=150, lr=0.05,
                       true_poses=true.astype(np.float64), ws=ws)
    assert res.loss[-1].mean() < 0.5 * res.loss[0].mean()
    assert np.all(res.rot_err_deg < rot0) and np.all(res.trans_err_mm < tr0)
    assert np.median(res.rot_err_deg) < np.median(rot0) / 3
    assert np.median(res.trans_err_mm) < np.median(tr0) / 3
    ws.close()
