"""The seeded synthetic inputs follow their stated recipe (phantom-derived
clouds, registration poses, detectors, uneven batches), and are reproducible:
the same seed gives the same bits. No GPU; the generators hold none of the
method's arithmetic, so these checks pin only the inputs both sides consume."""
import math

import numpy as np

from paper_2406_02518_gb300 import synthetic as syn


def _zyx_angles(R):
    """Angles (a, b, c) of R = Rz(a) Ry(b) Rx(c)."""
    b = -math.asin(max(-1.0, min(1.0, R[2, 0])))
    a = math.atan2(R[1, 0], R[0, 0])
    c = math.atan2(R[2, 1], R[2, 2])
    return a, b, c


def test_registration_workload_recipe():
    n, V, size, grid = 20_000, 8, 64, 64
    scene, views, st = syn.registration_workload(n, V, size, grid, seed=3)
    ph = syn.make_phantom(grid, 3)
    assert scene.n == n and scene.n_iso == n - n // 5
    # means: voxel centres inside the body ellipsoid, each voxel at most once
    vox = (scene.means.astype(np.float64) + ph.fov / 2) / ph.voxel - 0.5
    assert np.allclose(vox, np.rint(vox), atol=1e-3)
    body = np.array(ph.body_axes)
    assert np.all(np.sum((scene.means / body) ** 2, axis=1) <= 1.0 + 1e-6)
    assert np.unique(np.rint(vox), axis=0).shape[0] == n
    # log-scales log(voxel / 2) + U(-1/4, 1/4), unit quaternions
    d = scene.log_scales - math.log(ph.voxel / 2)
    assert d.min() >= -0.25 - 1e-6 and d.max() <= 0.25 + 1e-6 and d.std() > 0.1
    assert np.allclose(np.linalg.norm(scene.quats, axis=1), 1.0, atol=1e-6)
    # opacity from the phantom's HU at the mean
    hu = syn.phantom_hu(ph, scene.means.astype(np.float64))
    alpha = 1.0 / (1.0 + np.exp(-scene.opacity_logits.astype(np.float64)))
    assert np.allclose(alpha, np.clip(0.05 + 0.9 * (hu + 800.0) / 2300.0, 0.05, 0.95), atol=1e-5)
    # features: iso rows U(0, 1), dir rows N(0, 0.1^2); bases of the paper's k = 8, L = 1
    f_iso, f_dir = scene.feat[:scene.n_iso], scene.feat[scene.n_iso:]
    assert f_iso.min() >= 0.0 and f_iso.max() < 1.0 and abs(f_iso.mean() - 0.5) < 0.01
    assert abs(f_dir.std() - 0.1) < 0.005
    assert scene.b_iso.shape == (8,) and scene.B_dir.shape == (3, 8)
    # poses: rigid, Euler ZYX within +-15 deg and translations within +-20 mm of the AP view
    for T in views.world_to_cam.astype(np.float64):
        R, t = T[:, :3], T[:, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and abs(np.linalg.det(R) - 1) < 1e-6
        ang = np.degrees(_zyx_angles(syn.R_AP.T @ R))
        assert np.all(np.abs(ang) <= 15.0 + 1e-3)
        delta = syn.R_AP.T @ (t - np.array([0.0, 0.0, syn.SID_MM]))
        assert np.all(np.abs(delta) <= 20.0 + 1e-3)
    # detector: SDD 1020 mm, 256 mm wide, centred; near plane at a tenth of the SID
    assert np.allclose(views.detector, [[syn.SDD_MM, 256.0 / size, 256.0 / size, 0, 0]] * V)
    assert (views.height, views.width) == (size, size)
    assert abs(st.near_plane - 0.1 * syn.SID_MM) < 1e-9


def test_same_seed_same_bits():
    a = syn.registration_workload(5_000, 4, 32, 64, seed=7)
    b = syn.registration_workload(5_000, 4, 32, 64, seed=7)
    c = syn.registration_workload(5_000, 4, 32, 64, seed=8)
    for x, y, z in ((a[0].means, b[0].means, c[0].means), (a[0].feat, b[0].feat, c[0].feat),
                    (a[1].world_to_cam, b[1].world_to_cam, c[1].world_to_cam)):
        assert np.array_equal(x, y) and not np.array_equal(x, z)


def test_uneven_batch_recipe():
    scenes, views, _ = syn.uneven_workload(n_requests=3, seed=2)
    for sc, v in zip(scenes, views):
        assert 10_000 <= sc.n < 1_000_000 and sc.n_iso == sc.n - sc.n // 5
        assert v.n_views == 1 and v.height == v.width and v.height in (128, 256, 512, 1024)
        assert np.allclose(v.detector[0], [syn.SDD_MM, 256.0 / v.width, 256.0 / v.width, 0, 0])
