"""Radiodensity-aware dual sampling (RADS, Sec. 3.3) -- plain numpy oracle.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product library never imports or calls it, and it
calls nothing of the library.

What it computes, in the order of Sec. 3.3 and the implementation paragraph
of Sec. 4.1, on a CT volume of integer radiodensities (HU):

  P^mc  the marching-cubes points at the isolevel lambda = (min + max) / 2
        (the "average of the minimum and maximum volume"). Marching cubes puts
        one vertex on every edge of the voxel grid whose two end voxels lie on
        opposite sides of the isolevel, at the linear interpolation
        t = (lambda - f0) / (f1 - f0) along the edge; those vertices are the
        extracted interface points. n1 of them are kept, uniformly at random
        without replacement (all of them if there are fewer).
  P^dw  n2 voxel centroids drawn independently with probability proportional
        to the voxel's radiodensity above the volume's minimum, w = HU - min
        (the least dense voxel, air, weighs nothing).
  Isotropic Gaussians take all of P^mc and the first half of P^dw, the
  direction-dependent ones the second half (floor(n2 / 2) points).
  Scales follow the 3D Gaussian splatting default: isotropic, with
  log s = log sqrt(max(mean squared distance to the 3 nearest other points,
  1e-7)).

Randomness is counter-based so that any implementation reproduces it exactly:
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), whose output number i + 1 for seed s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15) with the published finaliser
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
  z ^ (z >> 31).
  - P^mc: edge e gets the key (splitmix64(seed, e) >> 32) << 32 | e; the n1
    smallest keys are kept (the low word makes keys distinct), listed in
    ascending edge order. Edge ids: 3 * voxel + axis, voxel = (z ny + y) nx + x,
    axis 0/1/2 for the +x/+y/+z neighbour.
  - P^dw: draw j takes u = splitmix64(~seed, j), target = floor(u * W / 2^64)
    with W the total weight, and the voxel whose cumulative-weight interval
    [C_{i-1}, C_i) holds the target; points are listed in draw order.
World position of voxel (x, y, z)'s centre: origin + spacing * (x, y, z).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * M1
    z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, idx) -> np.ndarray:
    """Output number idx + 1 of SplitMix64 seeded with `seed` (uint64 array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * GOLDEN
        return _mix(z)


def splitmix64_sequence(seed: int, n: int) -> list:
    """The generator run sequentially (state += golden gamma, then mix), in
    Python integers."""
    out, s = [], seed & MASK64
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out.append(z ^ (z >> 31))
    return out


def isolevel2(hu: np.ndarray) -> int:
    """2 * lambda = min + max (an integer, so the side test is exact)."""
    return int(hu.min()) + int(hu.max())


def mc_crossings(hu: np.ndarray, spacing, origin):
    """Marching-cubes vertices of the isolevel (min + max) / 2.

    hu: int [nz, ny, nx]. Returns (edge ids ascending [M] int64, world
    positions [M, 3] float64)."""
    hu = np.asarray(hu)
    nz, ny, nx = hu.shape
    lam2 = isolevel2(hu)
    above = 2 * hu.astype(np.int64) > lam2
    ids, pos = [], []
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = (zz * ny + yy) * nx + xx
    for axis, sl0, sl1 in ((0, np.s_[:, :, :-1], np.s_[:, :, 1:]),
                           (1, np.s_[:, :-1, :], np.s_[:, 1:, :]),
                           (2, np.s_[:-1, :, :], np.s_[1:, :, :])):
        cross = above[sl0] != above[sl1]
        f0 = hu[sl0][cross].astype(np.float64)
        f1 = hu[sl1][cross].astype(np.float64)
        t = (0.5 * lam2 - f0) / (f1 - f0)
        vox = np.stack([xx[sl0][cross], yy[sl0][cross], zz[sl0][cross]], 1).astype(np.float64)
        vox[:, axis] += t
        ids.append(3 * lin[sl0][cross].astype(np.int64) + axis)
        pos.append(vox)
    ids = np.concatenate(ids)
    pos = np.concatenate(pos)
    order = np.argsort(ids, kind="stable")
    p = pos[order] * np.asarray(spacing, np.float64) + np.asarray(origin, np.float64)
    return ids[order], p


def select_uniform(edge_ids: np.ndarray, n1: int, seed: int) -> np.ndarray:
    """Indices (into edge_ids) of the n1 kept crossings, in edge order."""
    e = np.asarray(edge_ids, np.int64)
    if e.size <= n1:
        return np.arange(e.size)
    key = (splitmix64(seed, e.astype(np.uint64)) >> np.uint64(32)) << np.uint64(32)
    key = key | e.astype(np.uint64)
    keep = np.argsort(key, kind="stable")[:n1]
    return np.sort(keep)


def weights(hu: np.ndarray) -> np.ndarray:
    """Radiodensity above the minimum, w = HU - min >= 0 (int64, voxel order)."""
    h = np.asarray(hu).astype(np.int64).reshape(-1)
    return h - h.min()


def draw_weighted(hu: np.ndarray, n2: int, seed: int) -> np.ndarray:
    """Voxel indices of n2 independent draws with P(i) = w_i / sum w. A volume
    with no weight at all (every voxel at the minimum) yields no draws."""
    w = weights(hu)
    cdf = np.cumsum(w)
    total = int(cdf[-1]) if cdf.size else 0
    if n2 <= 0 or total == 0:
        return np.zeros(0, np.int64)
    u = splitmix64(~seed & MASK64, np.arange(n2, dtype=np.uint64))
    target = np.array([(int(x) * total) >> 64 for x in u], dtype=np.int64)
    return np.searchsorted(cdf, target, side="right").astype(np.int64)


def voxel_centres(idx: np.ndarray, shape, spacing, origin) -> np.ndarray:
    nz, ny, nx = shape
    z, rem = np.divmod(np.asarray(idx, np.int64), ny * nx)
    y, x = np.divmod(rem, nx)
    v = np.stack([x, y, z], 1).astype(np.float64)
    return v * np.asarray(spacing, np.float64) + np.asarray(origin, np.float64)


def knn_log_scales(points: np.ndarray, k: int = 3, floor: float = 1e-7,
                   chunk: int = 256) -> np.ndarray:
    """log sqrt(max(mean of the k smallest squared distances to other points,
    floor)), by brute force over every pair (FP64). With fewer than k other
    points the mean runs over those there are; with none it is the floor."""
    p = np.asarray(points, np.float64)
    n = p.shape[0]
    out = np.empty(n)
    kk = min(k, n - 1)
    for s in range(0, n, chunk):
        q = p[s:s + chunk]
        d2 = np.zeros((q.shape[0], n))
        for a in range(3):
            d2 += (q[:, a, None] - p[None, :, a]) ** 2
        d2[np.arange(q.shape[0]), np.arange(s, s + q.shape[0])] = np.inf  # not itself
        if kk > 0:
            m = np.partition(d2, kk - 1, axis=1)[:, :kk].mean(axis=1)
        else:
            m = np.zeros(q.shape[0])
        out[s:s + chunk] = 0.5 * np.log(np.maximum(m, floor))
    return out


def rads(hu: np.ndarray, spacing, origin, n1: int = 15000, n2: int = 10000, seed: int = 0):
    """The whole initialisation: means [n, 3] (P^mc kept, then P^dw in draw
    order), isotropic log-scales [n], n_iso and the intermediate results."""
    edges, pos = mc_crossings(hu, spacing, origin)
    keep = select_uniform(edges, n1, seed)
    dw = draw_weighted(hu, n2, seed)
    p_dw = voxel_centres(dw, hu.shape, spacing, origin)
    means = np.concatenate([pos[keep], p_dw])
    return dict(means=means, log_scales=knn_log_scales(means), n_mc=int(keep.size),
                n_dw=int(dw.size), n_iso=int(keep.size) + (int(dw.size) - int(dw.size) // 2),
                edge_ids=edges[keep], n_crossings=int(edges.size), draw_voxels=dw,
                isolevel2=isolevel2(hu))
