"""ddgs_render_static: the forward render for callers that may not allocate
device memory while they run (fixed memory budgets, code inside another
runtime's allocator). Its scratch is a static device array; it must give the
same image, transmittance and list positions as ddgs_render.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import build
from paper_2406_02518_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4  # of the image range, as in the other GPU parity tests


def _call_static(lib, cloud, gv, cfg, out):
    g, v, c = cloud.struct(), gv.struct(), cfg.struct()
    img, tf, nl = out
    fn = lib.ddgs_render_static
    fn.argtypes = [C.c_void_p] * 7
    fn.restype = C.c_int32
    return fn(C.byref(g), C.byref(v), C.byref(c), img.data_ptr(), tf.data_ptr(), nl.data_ptr(),
              C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("seeds", [(11, 12)])
def test_static_render_matches_workspace_render_twice(seeds):
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    build.build()
    lib = B.load()
    ws = B.Workspace()
    for seed in seeds:  # two calls in a row share (and must reset) the scratch
        scene = syn.uniform_cloud(3000, seed=seed)
        views = syn.Views(np.ascontiguousarray(np.stack([
            syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])),
            syn.pose_matrix(syn.rot_y(0.4), np.array([0.0, 0.1, 2.2]))]).astype(np.float32)),
            syn.detector(2, 4.0, 8.0 / 100), 90, 100)
        cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
        cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
        ref_img, ref_tf, ref_nl = B.render(cloud, gv, cfg, ws)
        out = (torch.full_like(ref_img, -1.0), torch.full_like(ref_tf, -1.0),
               torch.full_like(ref_nl, -1))
        assert _call_static(lib, cloud, gv, cfg, out) == 0
        torch.cuda.synchronize()
        rng = float(ref_img.max() - ref_img.min())
        assert rng > 0.1
        assert float((out[0] - ref_img).abs().max()) <= IMG_TOL * rng
        assert float((out[1] - ref_tf).abs().max()) <= IMG_TOL * rng
        assert torch.equal(out[2], ref_nl)
    ws.close()


def test_static_render_rejects_oversized_inputs():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    build.build()
    lib = B.load()
    scene = syn.uniform_cloud(300_000, seed=1)  # 300k records > the 262144 limit
    views = syn.Views(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None].astype(np.float32),
                      syn.detector(1, 4.0, 8.0 / 64), 64, 64)
    cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
    cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
    out = (torch.zeros((1, 64, 64), device="cuda"), torch.zeros((1, 64, 64), device="cuda"),
           torch.zeros((1, 64, 64), dtype=torch.int32, device="cuda"))
    assert _call_static(lib, cloud, gv, cfg, out) == 2  # DDGS_ERR_CAPACITY
    assert float(out[0].abs().max()) == 0.0


_FRESH_PROCESS = r"""
import ctypes as C, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn
lib = B.load()
scene = syn.uniform_cloud(3000, seed=11)
views = syn.Views(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None].astype(np.float32),
                  syn.detector(1, 4.0, 8.0 / 100), 90, 100)
cloud, gv = B.cloud_from_arrays(scene), B.views_from_arrays(views)
cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
g, v, c = cloud.struct(), gv.struct(), cfg.struct()
img = torch.full((1, 90, 100), -1.0, device="cuda")
tf, nl = torch.empty_like(img), torch.empty((1, 90, 100), dtype=torch.int32, device="cuda")
fn = lib.ddgs_render_static
fn.argtypes = [C.c_void_p] * 7
fn.restype = C.c_int32
rc = fn(C.byref(g), C.byref(v), C.byref(c), img.data_ptr(), tf.data_ptr(), nl.data_ptr(),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
torch.cuda.synchronize()
if rc != 0:
    print("status", rc, lib.ddgs_last_cuda_error().decode())
    sys.exit(1)
np.save(sys.argv[2], img.cpu().numpy())
"""


def test_static_render_in_a_process_that_never_made_a_workspace(tmp_path):
    """The static entry point is the first and only library call of a process
    (no workspace has set up the binning kernels before it)."""
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "img.npy")
    r = subprocess.run([sys.executable, "-c", _FRESH_PROCESS, root, out], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-2000:]
    img = np.load(out)
    scene = syn.uniform_cloud(3000, seed=11)
    views = syn.Views(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None].astype(np.float32),
                      syn.detector(1, 4.0, 8.0 / 100), 90, 100)
    ws = B.Workspace()
    ref, _, _ = B.render(B.cloud_from_arrays(scene), B.views_from_arrays(views),
                         B.config_from_settings(syn.Settings(near_plane=0.2)), ws)
    ref = ref.cpu().numpy()
    ws.close()
    rng = float(ref.max() - ref.min())
    assert rng > 0.1
    assert float(np.abs(img - ref).max()) <= IMG_TOL * rng
