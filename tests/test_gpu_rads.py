"""GPU parity of the RADS initialisation (Sec. 3.3) against the oracle: the
crossing count, the kept edges and the drawn voxels bit for bit, positions to
binary32 rounding, scales against the oracle's neighbour search on the GPU's
own points."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import rads as R
from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2406_02518_gb300 import build
    build.build()
    B.load()
    assert B.device_supported(), "needs an sm_103 (GB300) device"


@pytest.fixture(scope="module")
def ws():
    w = B.Workspace()
    yield w
    w.close()


def _check(hu, spacing, origin, n1, n2, seed, ws, pos_tol=2e-4):
    g = B.rads(torch.as_tensor(hu, device="cuda"), spacing, origin, n1, n2, seed, ws=ws, debug=True)
    torch.cuda.synchronize()
    ref = R.rads(hu, spacing, origin, n1, n2, seed) if hu.size < 40 ** 3 or n1 + n2 < 6000 else None
    edges, pos = R.mc_crossings(hu, spacing, origin)
    keep = R.select_uniform(edges, n1, seed)
    draws = R.draw_weighted(hu, n2, seed)
    assert g["n_crossings"] == edges.size
    assert g["n_mc"] == keep.size and g["n_dw"] == draws.size
    assert g["n_iso"] == keep.size + draws.size - draws.size // 2
    assert np.array_equal(g["kept_edges"].cpu().numpy(), edges[keep])
    assert np.array_equal(g["draw_voxels"].cpu().numpy(), draws)
    means = g["means"].double().cpu().numpy()
    ref_means = np.concatenate([pos[keep], R.voxel_centres(draws, hu.shape, spacing, origin)])
    assert means.shape == ref_means.shape
    if means.size:
        assert np.abs(means - ref_means).max() <= pos_tol * max(1.0, np.abs(ref_means).max() / 100)
        ls = g["log_scales"].double().cpu().numpy()
        assert np.array_equal(ls[:, 0], ls[:, 1]) and np.array_equal(ls[:, 0], ls[:, 2])
        assert np.abs(ls[:, 0] - R.knn_log_scales(means)).max() < 2e-5
    if ref is not None and means.size:
        assert np.abs(means - ref["means"]).max() <= pos_tol * max(1.0, np.abs(ref_means).max() / 100)
    return g


@pytest.mark.parametrize("shape,seed", [((37, 29, 23), 0), ((5, 64, 130), 1), ((17, 3, 41), 2),
                                        ((37, 29, 24), 3), ((3, 5, 16), 4), ((2, 1, 8), 5),
                                        ((9, 70, 136), 6)])
def test_random_volumes(shape, seed, ws):
    """Rows of a multiple of 8 voxels take the 16-byte vector sweep; others the scalar one."""
    hu = np.random.default_rng(seed).integers(-1000, 2000, shape).astype(np.int16)
    _check(hu, (0.7, 1.1, 1.3), (-20.0, 5.0, 3.5), 500, 301, seed + 10, ws)


def test_phantom_volume_ragged_and_all_kept(ws):
    ph = syn.make_phantom(64, seed=3)
    hu = np.ascontiguousarray(syn.phantom_volume(ph)[3:61, 5:60, 1:63])  # 58 x 55 x 62
    sp, org = syn.volume_geometry(ph)
    g = _check(hu, sp, org, 1500, 1000, 4, ws)
    assert g["n_crossings"] > 1500
    g = _check(hu, sp, org, 10 ** 6, 40, 5, ws)  # n1 above the crossing count: every one kept
    assert g["n_mc"] == g["n_crossings"]


def test_degenerate_inputs(ws):
    # a uniform volume: no crossings, no weight, empty cloud
    g = _check(np.full((9, 10, 11), 40, np.int16), (1, 1, 1), (0, 0, 0), 100, 100, 0, ws)
    assert g["n_mc"] == g["n_dw"] == g["n_crossings"] == 0
    # single voxel, two voxels, n1 = 0, n2 = 0, voxel counts not a multiple of 8
    _check(np.array([[[5]]], np.int16), (1, 1, 1), (0, 0, 0), 10, 10, 1, ws)
    _check(np.array([[[-5, 7]]], np.int16), (2, 1, 1), (1, 0, 0), 10, 10, 1, ws)
    hu = np.random.default_rng(7).integers(-100, 100, (3, 5, 7)).astype(np.int16)
    _check(hu, (1, 1, 1), (0, 0, 0), 0, 50, 2, ws)
    _check(hu, (1, 1, 1), (0, 0, 0), 50, 0, 3, ws)


def test_invalid_volumes_are_rejected_on_the_host(ws):
    lib = B.load()
    buf = torch.zeros(64, dtype=torch.int16, device="cuda")
    out = torch.zeros((4, 3), device="cuda")
    counts = (C.c_int64 * 3)()

    def call(nx, ny, nz, ptr):
        vol = B._Volume(nx, ny, nz, ptr, (C.c_float * 3)(1, 1, 1), (C.c_float * 3)(0, 0, 0))
        return lib.ddgs_rads(C.byref(vol), 2, 2, C.c_uint64(0), ws.handle, B._ptr(out), B._ptr(out),
                             None, None, C.addressof(counts), B._stream())

    assert call(4, 4, 4, B._ptr(buf)) == 0
    assert call(4, 4, 4, B._ptr(buf) + 2) == 1            # not 16-byte aligned
    assert call(0, 4, 4, B._ptr(buf)) == 1                # empty axis
    assert call(2048, 1024, 1024, B._ptr(buf)) == 1       # edge ids beyond 32 bits
    torch.cuda.synchronize()


def test_paper_sizes_on_a_256_cube_phantom(ws):
    # Sec. 4.1: n1 = 15,000 marching-cubes points, n2 = 10,000 weighted draws
    ph = syn.make_phantom(256, seed=0)
    hu = syn.phantom_volume(ph)
    sp, org = syn.volume_geometry(ph)
    g = _check(hu, sp, org, 15000, 10000, 0, ws)
    assert g["n_mc"] == 15000 and g["n_dw"] == 10000 and g["n_iso"] == 20000
