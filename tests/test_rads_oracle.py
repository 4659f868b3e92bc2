"""Pins of the RADS oracle (Sec. 3.3): counter-based randomness, the
marching-cubes interface points, uniform and radiodensity-weighted sampling and
the nearest-neighbour scales, each against something other than the oracle's
own formulas (sequential generator runs, brute-force loops, closed-form
geometry, sampling statistics, scipy's KD-tree)."""
import math

import numpy as np
import pytest

from oracle import rads as R
from paper_2406_02518_gb300 import synthetic as syn


# ---- SplitMix64 ----

@pytest.mark.parametrize("seed", [0, 1, 1234567, 2**63 + 5, 2**64 - 1])
def test_counter_form_equals_sequential_generator(seed):
    n = 2000
    seq = R.splitmix64_sequence(seed, n)
    ctr = R.splitmix64(seed, np.arange(n, dtype=np.uint64))
    assert [int(x) for x in ctr] == seq


def test_published_splitmix64_outputs():
    # first outputs of the reference generator seeded with 1234567
    assert R.splitmix64_sequence(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_splitmix64_bytes_are_uniform():
    u = R.splitmix64(42, np.arange(1 << 16, dtype=np.uint64))
    for shift in (56, 32, 0):
        b = ((u >> np.uint64(shift)) & np.uint64(255)).astype(np.int64)
        cnt = np.bincount(b, minlength=256)
        chi2 = ((cnt - 256.0) ** 2 / 256.0).sum()
        assert chi2 < 255 + 6 * math.sqrt(2 * 255), (shift, chi2)


# ---- marching-cubes interface points ----

def _loops_crossings(hu):
    nz, ny, nx = hu.shape
    lam2 = int(hu.min()) + int(hu.max())
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for axis, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    X, Y, Z = x + dx, y + dy, z + dz
                    if X >= nx or Y >= ny or Z >= nz:
                        continue
                    a, b = int(hu[z, y, x]), int(hu[Z, Y, X])
                    if (2 * a > lam2) != (2 * b > lam2):
                        t = (lam2 / 2 - a) / (b - a)
                        out.append((3 * ((z * ny + y) * nx + x) + axis,
                                    x + t * dx, y + t * dy, z + t * dz))
    return out


@pytest.mark.parametrize("seed,shape", [(0, (5, 4, 3)), (1, (3, 7, 6)), (2, (1, 9, 2))])
def test_crossings_match_brute_force_loops(seed, shape):
    hu = np.random.default_rng(seed).integers(-1000, 1500, shape).astype(np.int16)
    ids, pos = R.mc_crossings(hu, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    ref = _loops_crossings(hu)
    assert ids.tolist() == [r[0] for r in ref]
    assert np.abs(pos - np.array([r[1:] for r in ref])).max() < 1e-12


def test_step_volume_gives_one_crossing_per_row_at_the_midpoint():
    nz, ny, nx, k = 4, 5, 9, 6
    hu = np.full((nz, ny, nx), -1000, np.int16)
    hu[:, :, k:] = 1000
    ids, pos = R.mc_crossings(hu, (0.5, 2.0, 3.0), (10.0, -4.0, 1.0))
    assert ids.size == nz * ny
    assert np.all(ids % 3 == 0)
    assert np.all(pos[:, 0] == 10.0 + 0.5 * (k - 0.5))


def test_ramp_crossings_lie_on_the_isoplane():
    z, y, x = np.meshgrid(np.arange(7), np.arange(8), np.arange(9), indexing="ij")
    hu = (x + 2 * y + 3 * z).astype(np.int16)  # linear: interpolation is exact
    ids, pos = R.mc_crossings(hu, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    lam = (int(hu.min()) + int(hu.max())) / 2
    assert ids.size > 50
    assert np.abs(pos[:, 0] + 2 * pos[:, 1] + 3 * pos[:, 2] - lam).max() < 1e-12


def test_sphere_crossing_count_follows_the_surface_area():
    # edges of a grid of spacing s crossing a surface number about
    # sum_a int |n_a| dA / s^2, i.e. 6 pi r^2 / s^2 for a sphere
    n, r, s = 64, 20.0, 1.0
    c = np.arange(n) - (n - 1) / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    hu = np.where(x * x + y * y + z * z <= r * r, 1000, -1000).astype(np.int16)
    ids, pos = R.mc_crossings(hu, (s, s, s), (0.0, 0.0, 0.0))
    expect = 6 * math.pi * r * r / (s * s)
    assert abs(ids.size / expect - 1) < 0.03
    rad = np.linalg.norm(pos - (n - 1) / 2, axis=1)
    assert np.abs(rad - r).max() < s


def test_isolevel_is_the_mid_range_and_the_side_test_exact():
    hu = np.array([[[-3, 0, 1, 4]]], np.int16)  # lambda = 0.5: 0 below, 1 above
    ids, pos = R.mc_crossings(hu, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    assert ids.tolist() == [3]  # only the edge 0 -> 1 (voxels 1 and 2)
    assert pos[0, 0] == 1.5


# ---- uniform subsample of P^mc ----

def test_selection_is_exact_size_sorted_and_uniform():
    edges = np.sort(np.random.default_rng(3).choice(10 ** 6, 200, replace=False))
    assert R.select_uniform(edges, 300, 0).tolist() == list(range(200))
    hits = np.zeros(200)
    trials = 2000
    for seed in range(trials):
        k = R.select_uniform(edges, 20, seed)
        assert k.size == 20 and np.all(np.diff(k) > 0)
        hits[k] += 1
    expect = trials * 20 / 200
    chi2 = ((hits - expect) ** 2 / expect).sum()
    assert chi2 < 199 + 6 * math.sqrt(2 * 199)


# ---- radiodensity-weighted draws ----

def _linear_scan(w, target):
    acc = 0
    for i, x in enumerate(w):
        acc += int(x)
        if acc > target:
            return i
    raise AssertionError("target beyond the total weight")


def test_draws_match_a_linear_scan_of_the_cumulative_weights():
    hu = np.random.default_rng(4).integers(-1000, 300, (3, 4, 5)).astype(np.int16)
    seed, n2 = 9, 300
    idx = R.draw_weighted(hu, n2, seed)
    w = R.weights(hu)
    total = int(w.sum())
    u = R.splitmix64_sequence(~seed & R.MASK64, n2)
    assert idx.tolist() == [_linear_scan(w, (x * total) >> 64) for x in u]


def test_draws_follow_the_weights():
    hu = np.full((2, 3, 4), -1000, np.int16)
    hu[0, 1, 2] = -999   # weight 1
    hu[1, 2, 3] = -997   # weight 3
    d = R.draw_weighted(hu, 20000, 5)
    a, b = (0 * 3 + 1) * 4 + 2, (1 * 3 + 2) * 4 + 3
    assert set(np.unique(d).tolist()) == {a, b}
    frac = np.mean(d == b)
    assert abs(frac - 0.75) < 4 * math.sqrt(0.75 * 0.25 / 20000)
    hu2 = np.random.default_rng(6).integers(-1000, 0, (4, 4, 4)).astype(np.int16)
    d2 = R.draw_weighted(hu2, 200000, 7)
    w = R.weights(hu2).astype(np.float64)
    cnt = np.bincount(d2, minlength=w.size)
    expect = 200000 * w / w.sum()
    m = expect > 0
    assert np.all(cnt[~m] == 0)
    chi2 = ((cnt[m] - expect[m]) ** 2 / expect[m]).sum()
    dof = int(m.sum()) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_uniform_volume_has_no_draws_and_no_crossings():
    hu = np.full((3, 3, 3), 40, np.int16)
    assert R.draw_weighted(hu, 10, 0).size == 0
    assert R.mc_crossings(hu, (1, 1, 1), (0, 0, 0))[0].size == 0


# ---- nearest-neighbour scales ----

def test_knn_scales_match_a_kd_tree():
    spatial = pytest.importorskip("scipy.spatial")
    p = np.random.default_rng(8).normal(size=(3000, 3)) * [1.0, 2.0, 0.5]
    ls = R.knn_log_scales(p)
    d, _ = spatial.cKDTree(p).query(p, 4)
    ref = 0.5 * np.log(np.maximum((d[:, 1:] ** 2).mean(1), 1e-7))
    assert np.abs(ls - ref).max() < 1e-12


def test_knn_scales_degenerate_sets():
    assert R.knn_log_scales(np.zeros((1, 3)))[0] == 0.5 * math.log(1e-7)
    two = np.array([[0.0, 0, 0], [3.0, 4.0, 0]])
    assert np.allclose(R.knn_log_scales(two), math.log(5.0))
    dup = np.zeros((5, 3))
    assert np.all(R.knn_log_scales(dup) == 0.5 * math.log(1e-7))


# ---- the whole initialisation on the phantom ----

def test_rads_on_the_phantom():
    ph = syn.make_phantom(48, seed=0)
    hu = syn.phantom_volume(ph)
    spacing, origin = syn.volume_geometry(ph)
    r = R.rads(hu, spacing, origin, n1=1500, n2=1001, seed=3)
    assert r["n_mc"] == 1500 and r["n_dw"] == 1001
    assert r["n_iso"] == 1500 + 501 and r["means"].shape == (2501, 3)
    # P^mc points sit on edges whose end voxels straddle the isolevel
    e = r["edge_ids"]
    vox, axis = e // 3, e % 3
    step = np.array([1, 48, 48 * 48])[axis]
    a, b = hu.reshape(-1)[vox].astype(int), hu.reshape(-1)[vox + step].astype(int)
    lam2 = r["isolevel2"]
    assert np.all((2 * a > lam2) != (2 * b > lam2))
    # P^dw points are centres of voxels denser than the minimum
    assert np.all(hu.reshape(-1)[r["draw_voxels"]] > hu.min())
    assert np.all(np.isfinite(r["log_scales"]))


def test_phantom_volume_equals_the_phantom_at_voxel_centres():
    n = 48
    ph = syn.make_phantom(n, seed=2, lesions=10)
    v = syn.phantom_volume(ph)
    c = (np.arange(n) + 0.5) * ph.voxel - ph.fov / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ref = syn.phantom_hu(ph, np.stack([x.ravel(), y.ravel(), z.ravel()], 1))
    assert np.array_equal(v, np.rint(ref).reshape(n, n, n).astype(np.int16))
