"""The radix sort's waits are bounded: a tile that never publishes its counts
makes the later tiles' waits run out, which the host reads as a timeout; the
context stays usable and the next render is exact again. No fault is made:
the hook only withholds a store, and every wait has an iteration limit."""
import numpy as np
import pytest
import torch

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

DDGS_ERR_TIMEOUT = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2406_02518_gb300 import build
    build.build()
    B.load()
    assert B.device_supported(), "needs an sm_103 (GB300) device"


def test_withheld_lookback_counts_time_out_and_are_reported():
    scene = syn.uniform_cloud(6000, seed=80)
    pose = syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None].astype(np.float32)
    views = syn.Views(pose, syn.detector(1, 4.0, 8.0 / 64), 64, 64)
    st = syn.Settings(near_plane=0.2, tile=8)
    cloud, gv, cfg = B.cloud_from_arrays(scene), B.views_from_arrays(views), B.config_from_settings(st)
    ws = B.Workspace()
    try:
        ref, _, _ = B.render(cloud, gv, cfg, ws)
        ref = ref.clone()
        assert ws.sync_status() == 0
        assert ws.pairs() > 2 * 4096  # several sort tiles, so later tiles wait on tile 0
        B.debug_withhold_tile(ws, 0)
        B.render(cloud, gv, cfg, ws)
        assert ws.sync_status() == DDGS_ERR_TIMEOUT
        B.debug_withhold_tile(ws, -1)
        img, _, _ = B.render(cloud, gv, cfg, ws)
        assert ws.sync_status() == 0
        torch.cuda.synchronize()
        assert torch.equal(img, ref)
    finally:
        B.debug_withhold_tile(ws, -1)
        ws.close()
