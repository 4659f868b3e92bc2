"""Pins of the oracle's FP32 binning reference (no GPU).

The binning is the integer part of the tiled renderer: which tiles a
Gaussian's q <= q_max ellipse reaches and the depth order inside each tile
(the order Eq. 1's product runs over). These tests check it against the FP64
projection of the oracle (every pixel with q <= q_max must lie in the
rectangle, and the rectangle must not be wider than the analytic ellipse
bound), and check the sorted list's invariants directly.
"""
import numpy as np
import pytest

import oracle
from paper_2406_02518_gb300 import synthetic as syn


def _case(n=600, seed=0, H=75, W=100, tile=16):
    sc = syn.uniform_cloud(n, seed=seed, log_scale_range=(-4.0, -1.5))
    views = syn.Views(np.ascontiguousarray(np.stack([
        syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])),
        syn.pose_matrix(syn.rot_y(0.4) @ syn.rot_x(-0.3), np.array([0.1, 0.0, 2.2]))
    ]).astype(np.float32)), syn.detector(2, 4.0, 8.0 / 96), H, W)
    return sc, views, syn.Settings(near_plane=0.2, tile=tile)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_rect_covers_every_pixel_inside_the_ellipse(tile):
    sc, views, st = _case(tile=tile)
    b = oracle.project32(sc, views, st)
    P = oracle.project64(sc, views, st)
    H, W = views.height, views.width
    jj, ii = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    n_in = 0
    for v in range(views.n_views):
        for i in range(sc.n):
            u, vv, ca, cb, cc, _, _, _, valid = P[v, i]
            dx, dy = u - jj, vv - ii
            q = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy
            inside = (q <= st.q_max) & (valid > 0)
            tt = b["tiles_touched"][v, i]
            if not inside.any():
                continue
            n_in += 1
            assert tt > 0
            r = b["rect"][v, i]
            rows, cols = np.nonzero(inside)
            assert (cols // tile).min() >= r[0] and (cols // tile).max() <= r[2]
            assert (rows // tile).min() >= r[1] and (rows // tile).max() <= r[3]
            assert tt == (r[2] - r[0] + 1) * (r[3] - r[1] + 1)
    assert n_in > 500


def test_rect_is_not_wider_than_the_ellipse_bound():
    sc, views, st = _case()
    b = oracle.project32(sc, views, st)
    P = oracle.project64(sc, views, st)
    H, W, t = views.height, views.width, st.tile
    for v in range(views.n_views):
        for i in range(sc.n):
            if b["tiles_touched"][v, i] == 0:
                continue
            u, vv, ca, cb, cc = P[v, i, :5]
            det = ca * cc - cb * cb
            ex = np.sqrt(st.q_max * cc / det) * 1.002 + 2e-3  # cov_a = conic_c / det
            ey = np.sqrt(st.q_max * ca / det) * 1.002 + 2e-3
            lo_c = max(int(np.ceil(u - ex - 0.5)), 0)
            hi_c = min(int(np.floor(u + ex - 0.5)), W - 1)
            lo_r = max(int(np.ceil(vv - ey - 0.5)), 0)
            hi_r = min(int(np.floor(vv + ey - 0.5)), H - 1)
            r = b["rect"][v, i]
            assert r[0] >= lo_c // t and r[2] <= hi_c // t
            assert r[1] >= lo_r // t and r[3] <= hi_r // t


def test_fp32_depth_agrees_with_fp64():
    sc, views, st = _case()
    b = oracle.project32(sc, views, st)
    P = oracle.project64(sc, views, st)
    z64 = P[:, :, 7]
    err = np.abs(b["depth"].astype(np.float64) - z64)
    assert (err <= 4 * np.spacing(b["depth"])).all()


def test_sorted_lists_invariants():
    sc, views, st = _case()
    r = oracle.bin32(sc, views, st)
    keys, vals, ranges = r["keys"], r["vals"], r["ranges"]
    assert r["m"] == int(r["tiles_touched"].sum()) > 0
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])  # stable: ties by index
    t = st.tile
    tx, ty = -(-views.width // t), -(-views.height // t)
    gt = (keys >> np.uint64(32)).astype(np.int64)
    v_of = gt // (tx * ty)
    local = gt % (tx * ty)
    # each pair's depth bits are its Gaussian's depth in that view
    d = r["depth"][v_of, vals.astype(np.int64)]
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), d.view(np.uint32))
    # each pair's tile lies in its Gaussian's rect, and each rect is fully listed
    rect = r["rect"][v_of, vals.astype(np.int64)]
    cx, cy = local % tx, local // tx
    assert np.all((cx >= rect[:, 0]) & (cx <= rect[:, 2]) & (cy >= rect[:, 1]) & (cy <= rect[:, 3]))
    counts = np.zeros(r["tiles_touched"].shape, np.int64)
    np.add.at(counts, (v_of, vals.astype(np.int64)), 1)
    assert np.array_equal(counts, r["tiles_touched"].astype(np.int64))
    # ranges
    for g in range(ranges.shape[0]):
        s, e = ranges[g]
        sel = np.flatnonzero(gt == g)
        if sel.size == 0:
            assert s == 0 and e == 0
        else:
            assert s == sel[0] and e == sel[-1] + 1


def test_culling_near_far_and_offscreen():
    sc = syn.uniform_cloud(50, seed=1)
    means = sc.means.copy()
    means[0] = [0, 0, -1.9]   # z = 0.1 < near (0.2)
    means[1] = [0, 0, 2.5]    # z = 4.5 > sdd (4)
    means[2] = [50, 0, 0]     # far off-screen
    sc.means = means
    views = syn.Views(syn._f32(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None]),
                      syn.detector(1, 4.0, 1 / 16), 128, 128)
    b = oracle.project32(sc, views, syn.Settings(near_plane=0.2))
    assert b["tiles_touched"][0, :3].tolist() == [0, 0, 0]
    assert b["tiles_touched"][0, 3:].min() > 0


def test_non_finite_geometry_is_culled():
    # a NaN depth, determinant, centre or extent fails the binning's comparisons
    sc = syn.uniform_cloud(50, seed=1)
    means, ls, qs = sc.means.copy(), sc.log_scales.copy(), sc.quats.copy()
    means[0] = [np.nan, 0, 0]       # NaN centre (and depth through the rotation)
    means[1, 0] = np.inf            # infinite centre
    ls[2] = [np.nan, -3, -3]        # NaN covariance
    qs[3] = [np.nan, 0, 0, 0]       # NaN rotation
    sc.means, sc.log_scales, sc.quats = means, ls, qs
    views = syn.Views(syn._f32(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None]),
                      syn.detector(1, 4.0, 1 / 16), 128, 128)
    b = oracle.project32(sc, views, syn.Settings(near_plane=0.2))
    assert b["tiles_touched"][0, :4].tolist() == [0, 0, 0, 0]
    assert b["tiles_touched"][0, 4:].min() > 0
