"""Seeded synthetic inputs for DRR splatting: Gaussian clouds, CT phantoms, poses.

This module only *generates inputs*; it holds none of the renderer's arithmetic
(no projection, radiosity or blending). Both the CUDA library and the CPU oracle
consume exactly these arrays, so the two see the same bits.

The paper's datasets (CTPelvic1K, NAF-CT, Ljubljana; Sec. 4.1) are not
available; ellipsoid CT phantoms stand in for them, at the paper's scale (clouds
of 10^4-10^6 Gaussians, CT grids up to 512^3, Sec. 4.2).

Conventions of the arrays (shared by definition with the library and oracle):
  means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z), opacity_logits [N],
  feat [N,k] (rows [0, n_iso) isotropic features, rows [n_iso, N)
  direction-dependent features), b_iso [k], B_dir [3,k] (degree L = 1).
  world_to_cam [V,3,4] rigid (R | t); detector [V,5] = (sdd, pitch_u, pitch_v,
  off_u, off_v); the source is the camera origin, the detector the plane
  z = sdd, pixel (row i, col j) has centre (j + 1/2, i + 1/2) in pixel units.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

K_FEAT = 8  # feature dimension k (Sec. 4.1: k = 8)
L_DEG = 1   # degree L of the direction decomposition (Sec. 4.1: L = 1)


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    feat: np.ndarray
    n_iso: int
    b_iso: np.ndarray
    B_dir: np.ndarray
    feat_dir_bf16: bool = False  # dir rows are exactly bf16-representable
    # Eq. 3 variants: every Gaussian carries both terms (direct-entangled,
    # Table 3); the ray angles are the pixel ray's rather than the mean's
    entangled: bool = False
    per_pixel: bool = False

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_dir(self) -> int:
        return self.n - self.n_iso


@dataclasses.dataclass
class Views:
    world_to_cam: np.ndarray
    detector: np.ndarray
    height: int
    width: int

    @property
    def n_views(self) -> int:
        return int(self.world_to_cam.shape[0])


@dataclasses.dataclass
class Settings:
    """Cutoffs and tiling of a render (values chosen where the paper is silent)."""
    near_plane: float
    tile: int = 16
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    q_max: float = 9.0


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return (b.astype(np.uint32)).view(np.float32)


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return _f32(q)


def logit(p: np.ndarray) -> np.ndarray:
    p = np.asarray(p, dtype=np.float64)
    return np.log(p) - np.log1p(-p)


def features(rng: np.random.Generator, n: int, n_iso: int, k: int = K_FEAT,
             dir_std: float = 0.1, bf16_dir: bool = False, sh_degree: int = L_DEG):
    """f_iso ~ U(0,1), f_dir ~ N(0, dir_std^2), b_iso [k], B_dir [L(L+2), k] ~ N(0,1)/sqrt(k)."""
    feat = np.empty((n, k), dtype=np.float32)
    feat[:n_iso] = rng.uniform(0.0, 1.0, (n_iso, k))
    feat[n_iso:] = rng.normal(0.0, dir_std, (n - n_iso, k))
    if bf16_dir:
        feat[n_iso:] = round_to_bf16(feat[n_iso:])
    b_iso = _f32(rng.standard_normal(k) / math.sqrt(k))
    B_dir = _f32(rng.standard_normal((sh_degree * (sh_degree + 2), k)) / math.sqrt(k))
    return feat, b_iso, B_dir


# --------------------------------------------------------------------------
# Poses
# --------------------------------------------------------------------------

def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


# Anterior-posterior base view: camera z (beam direction) = world +y,
# camera x = world x, camera y = world -z.
R_AP = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def pose_matrix(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    T = np.zeros((3, 4), dtype=np.float64)
    T[:, :3] = R
    T[:, 3] = t
    return T


def registration_poses(rng: np.random.Generator, n_views: int, sid: float,
                       max_deg: float = 15.0, max_mm: float = 20.0) -> np.ndarray:
    """Candidate poses about the isocenter: Euler ZYX angles U(-max_deg, max_deg),
    translations U(-max_mm, max_mm) per axis, composed on the AP view."""
    out = np.zeros((n_views, 3, 4), dtype=np.float64)
    for v in range(n_views):
        a, b, c = np.deg2rad(rng.uniform(-max_deg, max_deg, 3))
        Rp = rot_z(a) @ rot_y(b) @ rot_x(c)
        delta = rng.uniform(-max_mm, max_mm, 3)
        R = R_AP @ Rp
        t = R_AP @ delta + np.array([0.0, 0.0, sid])
        out[v] = pose_matrix(R, t)
    return _f32(out)


def ap_pose(sid: float) -> np.ndarray:
    return _f32(pose_matrix(R_AP, np.array([0.0, 0.0, sid]))[None])


def orbit_poses(n_views: int, sid: float, step_deg: float = 45.0) -> np.ndarray:
    """Circular orbit about world z, step_deg apart, starting at AP."""
    out = np.zeros((n_views, 3, 4), dtype=np.float64)
    for v in range(n_views):
        R = R_AP @ rot_z(-np.deg2rad(step_deg * v))
        out[v] = pose_matrix(R, np.array([0.0, 0.0, sid]))
    return _f32(out)


def detector(n_views: int, sdd: float, pitch: float, off=(0.0, 0.0)) -> np.ndarray:
    d = np.zeros((n_views, 5), dtype=np.float32)
    d[:, 0] = sdd
    d[:, 1] = pitch
    d[:, 2] = pitch
    d[:, 3] = off[0]
    d[:, 4] = off[1]
    return d


# --------------------------------------------------------------------------
# Uniform cloud (the 4,096-Gaussian plain forward workload)
# --------------------------------------------------------------------------

def uniform_cloud(n: int = 4096, seed: int = 0, k: int = K_FEAT,
                  dir_frac: float = 0.2, extent: float = 1.0,
                  log_scale_range=(-4.0, -2.0), alpha_range=(0.1, 0.9),
                  dir_std: float = 0.1, sh_degree: int = L_DEG) -> Scene:
    """Means U[-extent, extent]^3, log-scales U(range), uniform unit quaternions,
    alpha U(range) stored as logits, f_iso U(0,1), f_dir N(0, dir_std^2);
    the last floor(dir_frac * n) Gaussians are direction-dependent."""
    rng = np.random.default_rng(seed)
    n_dir = int(math.floor(dir_frac * n))
    means = _f32(rng.uniform(-extent, extent, (n, 3)))
    log_scales = _f32(rng.uniform(log_scale_range[0], log_scale_range[1], (n, 3)))
    quats = random_quats(rng, n)
    alpha = rng.uniform(alpha_range[0], alpha_range[1], n)
    feat, b_iso, B_dir = features(rng, n, n - n_dir, k, dir_std, sh_degree=sh_degree)
    return Scene(means, log_scales, quats, _f32(logit(alpha)), feat, n - n_dir,
                 b_iso, B_dir)


def plain_forward_workload(seed: int = 0, n: int = 4096, size: int = 128):
    """4,096 Gaussians in [-1,1]^3, one cone-beam view: source-to-isocenter 2,
    source-to-detector 4, 128 x 128 detector of 8 x 8 units."""
    scene = uniform_cloud(n, seed)
    views = Views(_f32(pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))[None]),
                  detector(1, 4.0, 8.0 / size), size, size)
    return scene, views, Settings(near_plane=0.2)


# --------------------------------------------------------------------------
# CT phantom (nested ellipsoids) and Gaussian initialisation from it
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Phantom:
    n: int                 # grid size n^3
    voxel: float           # mm
    structures: list       # (kind, centre[3], axes[3], R[3,3], hu, wall)
    body_axes: tuple = (100.0, 80.0, 120.0)
    body_hu: float = 40.0

    @property
    def fov(self) -> float:
        return self.n * self.voxel


def make_phantom(n: int, seed: int = 0, fov: float = 256.0,
                 lesions: int = 0) -> Phantom:
    """Air -1000 HU; body ellipsoid (100, 80, 120) mm of soft tissue U(0, 80) HU;
    6 organ ellipsoids (U(0,80) HU, semi-axes 15-40 mm); 4 bone shells
    (hollow ellipsoids, 5 mm wall, U(400,1500) HU, semi-axes 20-60 mm); optional
    spherical lesions (radius U(3,15) mm, +U(30,100) HU over their host)."""
    rng = np.random.default_rng(seed)
    body = np.array([100.0, 80.0, 120.0])
    structs = []

    def place(axes):
        lim = np.maximum(body - axes, 5.0) * 0.6
        return rng.uniform(-lim, lim)

    for _ in range(6):
        axes = rng.uniform(15, 40, 3)
        R = rot_z(rng.uniform(0, 2 * math.pi)) @ rot_y(rng.uniform(0, math.pi)) @ rot_x(rng.uniform(0, 2 * math.pi))
        structs.append(("organ", place(axes), axes, R, rng.uniform(0, 80), 0.0))
    for _ in range(4):
        axes = rng.uniform(20, 60, 3)
        R = rot_z(rng.uniform(0, 2 * math.pi)) @ rot_y(rng.uniform(0, math.pi)) @ rot_x(rng.uniform(0, 2 * math.pi))
        structs.append(("bone", place(axes), axes, R, rng.uniform(400, 1500), 5.0))
    for _ in range(lesions):
        r = rng.uniform(3, 15)
        structs.append(("lesion", place(np.array([r, r, r])), np.array([r, r, r]),
                        np.eye(3), rng.uniform(30, 100), 0.0))
    return Phantom(n, fov / n, structs, tuple(body), float(rng.uniform(0, 80)))


def _apply_structure(hu: np.ndarray, pts: np.ndarray, inside: np.ndarray, st) -> np.ndarray:
    kind, c, axes, R, val, wall = st
    loc = (pts - c) @ R  # coordinates in the structure frame
    r2 = np.sum((loc / axes) ** 2, axis=1)
    if kind == "bone":
        inner = np.maximum(axes - wall, 1.0)
        m = (r2 <= 1.0) & (np.sum((loc / inner) ** 2, axis=1) > 1.0) & inside
        return np.where(m, val, hu)
    if kind == "organ":
        return np.where((r2 <= 1.0) & inside, val, hu)
    return np.where((r2 <= 1.0) & inside, hu + val, hu)  # lesion: additive over its host


def phantom_hu(ph: Phantom, pts: np.ndarray) -> np.ndarray:
    """HU at world points pts [M,3] (mm, isocenter at the origin)."""
    body = np.array(ph.body_axes)
    inside = np.sum((pts / body) ** 2, axis=1) <= 1.0
    hu = np.where(inside, ph.body_hu, -1000.0)
    for st in ph.structures:
        hu = _apply_structure(hu, pts, inside, st)
    return hu


def voxel_centres(ph: Phantom, flat_idx: np.ndarray) -> np.ndarray:
    n = ph.n
    iz, rem = np.divmod(flat_idx, n * n)
    iy, ix = np.divmod(rem, n)
    idx = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    return (idx + 0.5) * ph.voxel - ph.fov / 2


def phantom_volume(ph: Phantom) -> np.ndarray:
    """The phantom sampled at its voxel centres as a CT volume: int16 HU,
    [z][y][x] with x fastest. Same values as phantom_hu at the centres; each
    structure is evaluated only on the points of a box around its bounding
    sphere (it cannot change any other point)."""
    n = ph.n
    c = (np.arange(n) + 0.5) * ph.voxel - ph.fov / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")
    body = np.array(ph.body_axes)
    out = np.empty((n, n, n), np.int16)
    for iz in range(n):
        pts = np.stack([xx.ravel(), yy.ravel(), np.full(n * n, c[iz])], 1)
        inside = np.sum((pts / body) ** 2, axis=1) <= 1.0
        hu = np.where(inside, ph.body_hu, -1000.0)
        for st in ph.structures:
            ctr, r = st[1], float(np.max(st[2])) * 1.001 + ph.voxel
            if abs(c[iz] - ctr[2]) > r:
                continue
            sel = np.flatnonzero((np.abs(pts[:, 0] - ctr[0]) <= r) & (np.abs(pts[:, 1] - ctr[1]) <= r))
            if sel.size:
                hu[sel] = _apply_structure(hu[sel], pts[sel], inside[sel], st)
        out[iz] = np.clip(np.rint(hu), -32768, 32767).reshape(n, n)
    return out


def volume_geometry(ph: Phantom):
    """(spacing, origin) of phantom_volume: voxel size per axis and the world
    position of voxel (0, 0, 0)'s centre, mm."""
    v = float(ph.voxel)
    o = -ph.fov / 2 + 0.5 * v
    return (v, v, v), (o, o, o)


def body_voxels(ph: Phantom) -> np.ndarray:
    """Flat indices of the voxels whose HU exceeds -800 (the body ellipsoid)."""
    n = ph.n
    c = (np.arange(n) + 0.5) * ph.voxel - ph.fov / 2
    bx, by, bz = ph.body_axes
    yy, xx = np.meshgrid(c, c, indexing="ij")
    base = (xx / bx) ** 2 + (yy / by) ** 2
    out = []
    for iz in range(n):
        rz = (c[iz] / bz) ** 2
        if rz > 1.0:
            continue
        sl = np.flatnonzero((base + rz) <= 1.0)
        out.append(sl + iz * n * n)
    return np.concatenate(out).astype(np.int64)


def gaussians_from_phantom(ph: Phantom, n_gauss: int, seed: int = 0,
                           k: int = K_FEAT, dir_frac: float = 0.2,
                           bf16_dir: bool = False, candidates=None,
                           sh_degree: int = L_DEG) -> Scene:
    """One candidate per voxel above -800 HU, subsampled without replacement to
    n_gauss. mu = voxel centre; log_s = log(voxel/2) + U(-1/4, 1/4);
    uniform unit quaternions; alpha = clip(0.05 + 0.9 (HU + 800) / 2300, 0.05,
    0.95) as a logit; the last floor(dir_frac n) Gaussians (a seeded random
    subset) are direction-dependent. `candidates` (body_voxels(ph)) may be
    passed in when many clouds come from one phantom."""
    rng = np.random.default_rng(seed)
    cand = body_voxels(ph) if candidates is None else candidates
    if n_gauss > cand.size:
        raise ValueError(f"phantom has only {cand.size} voxels above -800 HU")
    pick = np.sort(rng.choice(cand.size, n_gauss, replace=False))
    pick = rng.permutation(cand[pick])  # the permutation decides iso vs dir
    mu = voxel_centres(ph, pick)
    hu = phantom_hu(ph, mu)
    n_dir = int(math.floor(dir_frac * n_gauss))
    log_s = np.log(0.5 * ph.voxel) + rng.uniform(-0.25, 0.25, (n_gauss, 3))
    quats = random_quats(rng, n_gauss)
    alpha = np.clip(0.05 + 0.9 * (hu + 800.0) / 2300.0, 0.05, 0.95)
    feat, b_iso, B_dir = features(rng, n_gauss, n_gauss - n_dir, k, 0.1, bf16_dir, sh_degree)
    return Scene(_f32(mu), _f32(log_s), quats, _f32(logit(alpha)), feat,
                 n_gauss - n_dir, b_iso, B_dir, bf16_dir)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

SDD_MM = 1020.0
SID_MM = 816.0


def registration_workload(n_gauss: int = 500_000, n_views: int = 64,
                          size: int = 256, grid: int = 256, seed: int = 0):
    """Batched pose registration: Gaussians from a 256^3 phantom (1 mm voxels),
    64 candidate poses (+-15 deg, +-20 mm), 256^2 detector of 1 mm pitch,
    source-to-detector 1020 mm, source-to-isocenter 816 mm."""
    ph = make_phantom(grid, seed)
    scene = gaussians_from_phantom(ph, n_gauss, seed)
    rng = np.random.default_rng(seed + 1000)
    views = Views(registration_poses(rng, n_views, SID_MM),
                  detector(n_views, SDD_MM, 256.0 / size), size, size)
    return scene, views, Settings(near_plane=0.1 * SID_MM)


def fit_workload(n_gauss: int = 100_000, size: int = 512, grid: int = 128, seed: int = 0):
    """Forward+backward fit step: Gaussians from a 128^3 phantom (2 mm voxels),
    one AP view, 512^2 detector at 0.5 mm pitch, SDD 1020 mm, SID 816 mm."""
    ph = make_phantom(grid, seed)
    scene = gaussians_from_phantom(ph, n_gauss, seed)
    views = Views(ap_pose(SID_MM), detector(1, SDD_MM, 256.0 / size), size, size)
    return scene, views, Settings(near_plane=0.1 * SID_MM)


def large_fit_workload(n_gauss: int = 2_000_000, size: int = 1024, grid: int = 512,
                       n_views: int = 8, seed: int = 0):
    """Large fit: 512^3 phantom (0.5 mm) with 20 lesions, 8 orbit views at 45
    degrees, 1024^2 detector at 0.25 mm, direction-dependent features in bf16."""
    ph = make_phantom(grid, seed, lesions=20)
    scene = gaussians_from_phantom(ph, n_gauss, seed, bf16_dir=True)
    views = Views(orbit_poses(n_views, SID_MM), detector(n_views, SDD_MM, 256.0 / size),
                  size, size)
    return scene, views, Settings(near_plane=0.1 * SID_MM)


def uneven_workload(n_requests: int = 256, grid: int = 512, seed: int = 0,
                    log10_range=(4.0, 6.0), sizes=(128, 256, 512, 1024)):
    """Uneven batch: n_requests clouds of floor(10^U(4, 6)) Gaussians, each
    subsampled from one 512^3 phantom (0.5 mm voxels, with lesions), each with
    one view: a detector side drawn from `sizes` (pitch 256/side mm) and a
    registration pose (+-15 deg, +-20 mm) about the isocenter."""
    ph = make_phantom(grid, seed, lesions=20)
    cand = body_voxels(ph)
    rng = np.random.default_rng(seed + 7)
    scenes, views = [], []
    for r in range(n_requests):
        n = int(10 ** rng.uniform(*log10_range))
        scenes.append(gaussians_from_phantom(ph, n, seed=seed + 100 + r, candidates=cand))
        side = int(rng.choice(sizes))
        views.append(Views(registration_poses(rng, 1, SID_MM), detector(1, SDD_MM, 256.0 / side),
                           side, side))
    return scenes, views, Settings(near_plane=0.1 * SID_MM)


def perturb_scene(scene: Scene, seed: int = 1, mu_mm: float = 1.0,
                  logit_std: float = 0.2) -> Scene:
    """The fit target's scene: means + N(0, mu_mm^2), logits + N(0, logit_std^2)."""
    rng = np.random.default_rng(seed)
    return dataclasses.replace(
        scene,
        means=_f32(scene.means + rng.normal(0, mu_mm, scene.means.shape)),
        opacity_logits=_f32(scene.opacity_logits + rng.normal(0, logit_std, scene.n)))


def sample_pixels(views: Views, n_random: int = 4096, n_rows: int = 4,
                  seed: int = 0, view_ids=None) -> np.ndarray:
    """Seeded pixel subset per view: n_random uniform pixels plus n_rows full
    rows. Returns int32 [M,3] = (view, row, col), unique, sorted."""
    rng = np.random.default_rng(seed)
    H, W = views.height, views.width
    out = []
    for v in (range(views.n_views) if view_ids is None else view_ids):
        r = rng.integers(0, H, n_random)
        c = rng.integers(0, W, n_random)
        rows = rng.choice(H, min(n_rows, H), replace=False)
        rr = np.repeat(rows, W)
        cc = np.tile(np.arange(W), len(rows))
        p = np.stack([np.full(n_random + rr.size, v), np.concatenate([r, rr]),
                      np.concatenate([c, cc])], axis=1)
        out.append(np.unique(p, axis=0))
    return np.ascontiguousarray(np.concatenate(out).astype(np.int32))
