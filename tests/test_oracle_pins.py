"""Pins of the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a worked example printed in the paper, a brute-force evaluation, an
invariance, a special case that reduces to a simpler model, or finite
differences. A plausible mistake anywhere in the oracle (a transposed pose, a
wrong Jacobian sign, a dropped transmittance factor, a wrong harmonic) fails at
least one of them.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2406_02518_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(means, log_scales, quats, logits, feat, n_iso, b_iso=None, B_dir=None):
    k = feat.shape[1]
    b_iso = np.ones(k, np.float32) if b_iso is None else b_iso
    B_dir = np.zeros((3, k), np.float32) if B_dir is None else B_dir
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return syn.Scene(f(means), f(log_scales), f(quats), f(logits), f(feat), n_iso, f(b_iso),
                     f(B_dir))


def _views(poses, sdd, pitch, H, W, off=(0.0, 0.0)):
    poses = np.asarray(poses, np.float32).reshape(-1, 3, 4)
    return syn.Views(np.ascontiguousarray(poses), syn.detector(poses.shape[0], sdd, pitch, off),
                     H, W)


def _pose(R, t):
    return syn.pose_matrix(np.asarray(R, np.float64), np.asarray(t, np.float64))


# ---------------------------------------------------------------------------
# exp in binary32 used by the FP32 binning reference
# ---------------------------------------------------------------------------

def test_exp32_within_two_ulp_of_exp():
    xs = np.concatenate([np.linspace(-20, 20, 4001), np.array([0.0, -1e-8, 1e-8, 1.0, -1.0])])
    for x in xs.astype(np.float32):
        got = oracle.exp32(float(x))
        ref = math.exp(float(x))
        ulp = np.spacing(np.float32(ref))
        assert abs(got - ref) <= 2 * ulp, (x, got, ref)
    assert oracle.exp32(0.0) == 1.0


# ---------------------------------------------------------------------------
# Projection: the closed-form line integral of one 3D Gaussian
# ---------------------------------------------------------------------------

def _line_integral_ratio(Sigma, mu, src, dirs, dstar):
    """L(p) / L(p*) for rays src + t d: exact integral of exp(-x^T Sigma^-1 x / 2)."""
    Si = np.linalg.inv(Sigma)
    m = src - mu

    def logL(d):
        # exponent m^T Si m - (d^T Si m)^2 / (d^T Si d), evaluated as the
        # Si-norm of m with its Si-projection on d removed (no cancellation)
        a = d @ Si @ d
        mp = m - d * ((d @ Si @ m) / a)
        return 0.5 * math.log(2 * math.pi / a) - 0.5 * (mp @ Si @ mp)

    l0 = logL(dstar)
    return np.array([math.exp(logL(d) - l0) for d in dirs])


def _single_gaussian_profile(sid, sdd, scale, rng, H=33, W=33):
    """One isotropic Gaussian near the isocenter (dilation 0). Returns the
    oracle's G = C / (c alpha) and the exact line-integral ratio per pixel."""
    rot = Rotation.random(random_state=rng)
    qxyzw = rot.as_quat()
    quat = np.array([qxyzw[3], qxyzw[0], qxyzw[1], qxyzw[2]])
    s = scale * np.array([1.0, 1.7, 0.6])
    mu = np.array([0.3, -0.2, 0.1]) * scale
    R_cam = Rotation.random(random_state=rng).as_matrix()
    t = np.array([0.0, 0.0, sid]) - R_cam @ np.zeros(3)
    mag = sdd / sid
    pitch = mag * scale / 3.0  # the Gaussian spans roughly 10 pixels
    views = _views(_pose(R_cam, t), sdd, pitch, H, W)
    scene = _scene(mu[None], np.log(s)[None], quat[None], [0.0], np.zeros((1, 8)), 1)
    st = syn.Settings(near_plane=0.1 * sid, dilation=0.0, alpha_min=1e-12, t_min=1e-12,
                      q_max=9.0)
    r = oracle.render(scene, views, st)
    # c = sigmoid(0) = 0.5, alpha = sigmoid(0) = 0.5, T = 1: C = 0.25 G
    G = r["image"][0] / 0.25
    # exact ratio from the float32 inputs the oracle saw
    mu32 = scene.means[0].astype(np.float64)
    R32 = views.world_to_cam[0, :, :3].astype(np.float64)
    t32 = views.world_to_cam[0, :, 3].astype(np.float64)
    q32 = scene.quats[0].astype(np.float64)
    Rg = Rotation.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()
    Sigma = Rg @ np.diag(np.exp(2 * scene.log_scales[0].astype(np.float64))) @ Rg.T
    # the camera map x -> W x + t of the (float32-rounded, so not exactly
    # orthogonal) pose: rays leave W^-1 (-t) along W^-1 cam
    Wi = np.linalg.inv(R32)
    src = -Wi @ t32
    det = views.detector[0].astype(np.float64)
    fu, fv = det[0] / det[1], det[0] / det[2]
    cu, cv = W / 2 + det[3], H / 2 + det[4]
    jj, ii = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    cam = np.stack([(jj - cu) / fu, (ii - cv) / fv, np.ones_like(jj)], -1).reshape(-1, 3)
    dirs = cam @ Wi.T
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dstar = (mu32 - src) / np.linalg.norm(mu32 - src)
    ratio = _line_integral_ratio(Sigma, mu32, src, dirs, dstar).reshape(H, W)
    inside = G > 0
    return G, ratio, inside


def test_projection_matches_line_integral_orthographic_limit():
    rng = np.random.default_rng(11)
    G, ratio, inside = _single_gaussian_profile(sid=1e6, sdd=2e6, scale=1.0, rng=rng)
    assert inside.sum() > 40
    err = np.abs(G - ratio)[inside].max()
    assert err < 2e-6, err


def test_projection_error_shrinks_with_scale_over_depth():
    errs = []
    for sd in (1e-1, 1e-2, 1e-3):
        rng = np.random.default_rng(5)
        G, ratio, inside = _single_gaussian_profile(sid=1.0, sdd=2.0, scale=sd, rng=rng)
        assert inside.sum() > 40
        errs.append(np.abs(G - ratio)[inside].max())
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs


# ---------------------------------------------------------------------------
# Eq. 1 compositing: worked example, Beer-Lambert, brute-force order
# ---------------------------------------------------------------------------

def _coaxial_scene(alphas, colors_logit, depths):
    n = len(alphas)
    means = np.zeros((n, 3))
    means[:, 2] = depths
    feat = np.zeros((n, 8))
    feat[:, 0] = colors_logit  # b_iso = e_0: c = sigmoid(f_0)
    b = np.zeros(8)
    b[0] = 1.0
    scene = _scene(means, np.full((n, 3), math.log(0.05)), np.tile([1.0, 0, 0, 0], (n, 1)),
                   syn.logit(np.array(alphas)), feat, n, b_iso=b)
    views = _views(_pose(np.eye(3), [0.0, 0.0, 2.0]), 4.0, 0.05, 3, 3)
    return scene, views


def test_worked_example_two_half_attenuations():
    g = json.load(open(os.path.join(GOLDEN, "beer_lambert_two_layers.json")))
    a1, a2 = g["attenuations"]
    scene, views = _coaxial_scene([a1, a2], [0.3, -0.7], [-0.2, 0.4])
    st = syn.Settings(near_plane=0.2, dilation=0.0)
    r = oracle.render(scene, views, st)
    T = r["t_final"][0, 1, 1]  # centre pixel: q = 0 for both
    assert abs((1 - T) - g["total_attenuation"]) < 1e-12
    f0 = scene.feat[:, 0].astype(np.float64)  # float32-rounded colour logits
    c1, c2 = 1 / (1 + math.exp(-f0[0])), 1 / (1 + math.exp(-f0[1]))
    assert abs(r["image"][0, 1, 1] - (c1 * a1 + c2 * a2 * (1 - a1))) < 1e-12
    assert r["n_contrib"][0, 1, 1] == 2


def test_transmittance_is_beer_lambert():
    # sigma_l = 1 - exp(-a_l delta_l) (Appendix A.1, Eq. 5): T = exp(-sum a delta)
    ad = np.array([0.3, 0.05, 1.1, 0.4])
    alphas = 1 - np.exp(-ad)
    scene, views = _coaxial_scene(alphas, [0.0] * 4, [-0.5, -0.1, 0.2, 0.6])
    st = syn.Settings(near_plane=0.2, dilation=0.0, alpha_max=0.999)
    T = oracle.render(scene, views, st)["t_final"][0, 1, 1]
    # logits are float32-rounded: compare with the alphas the oracle saw
    a32 = 1 / (1 + np.exp(-scene.opacity_logits.astype(np.float64)))
    assert abs(T - np.prod(1 - a32)) < 1e-14
    assert abs(T - math.exp(-ad.sum())) < 1e-6


def _brute_force_image(scene, views, st):
    """Eq. 1 with T_j = prod over Gaussians strictly in front of j, no sort."""
    P = oracle.project64(scene, views, st)
    V, H, W = views.n_views, views.height, views.width
    img = np.zeros((V, H, W))
    for v in range(V):
        u, vv, ca, cb, cc, al, col, z, valid = P[v].T
        for i in range(H):
            for j in range(W):
                dx, dy = u - (j + 0.5), vv - (i + 0.5)
                q = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy
                sig = np.minimum(st.alpha_max, al * np.exp(-0.5 * q))
                use = (valid > 0) & (q <= st.q_max) & (sig >= st.alpha_min)
                acc = 0.0
                for a in np.flatnonzero(use):
                    front = use & ((z < z[a]) | ((z == z[a]) & (np.arange(len(z)) < a)))
                    acc += col[a] * sig[a] * np.prod(1 - sig[front])
                img[v, i, j] = acc
    return img


def test_compositing_matches_brute_force_order():
    sc = syn.uniform_cloud(8, seed=3, extent=0.5, log_scale_range=(-2.0, -1.2),
                           alpha_range=(0.3, 0.9))
    views = _views(_pose(np.eye(3), [0.0, 0.0, 2.0]), 4.0, 0.25, 12, 10)
    st = syn.Settings(near_plane=0.2, t_min=1e-30, alpha_min=1e-30, q_max=1e4)
    got = oracle.render(sc, views, st)["image"]
    ref = _brute_force_image(sc, views, st)
    assert np.abs(got - ref).max() < 1e-13
    assert ref.max() > 0.1


def test_storage_permutation_invariance():
    sc = syn.uniform_cloud(300, seed=4)
    views = _views(_pose(np.eye(3), [0.0, 0.0, 2.0]), 4.0, 1 / 8, 64, 48)
    st = syn.Settings(near_plane=0.2)
    base = oracle.render(sc, views, st)
    rng = np.random.default_rng(0)
    perm = np.concatenate([rng.permutation(sc.n_iso), sc.n_iso + rng.permutation(sc.n_dir)])
    sp = dataclasses.replace(sc, means=sc.means[perm].copy(), log_scales=sc.log_scales[perm].copy(),
                             quats=sc.quats[perm].copy(), opacity_logits=sc.opacity_logits[perm].copy(),
                             feat=sc.feat[perm].copy())
    r = oracle.render(sp, views, st)
    assert np.abs(r["image"] - base["image"]).max() < 1e-13
    ok = base["last_id"] >= 0
    assert np.array_equal(perm[r["last_id"][ok]], base["last_id"][ok])


# ---------------------------------------------------------------------------
# Invariance under a joint rigid motion of scene and cameras
# ---------------------------------------------------------------------------

_A = np.array([[0.0, -1.0, 0.0], [0.0, 0.0, 1.0], [-1.0, 0.0, 0.0]])  # Y_1 = C1 * A d


def _move(scene, views, Q, s):
    qQ = Rotation.from_matrix(Q)
    q = scene.quats.astype(np.float64)
    rq = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1))
    qn = (qQ * rq).as_quat()
    quats = np.stack([qn[:, 3], qn[:, 0], qn[:, 1], qn[:, 2]], 1)
    means = scene.means.astype(np.float64) @ Q.T + s
    T = views.world_to_cam.astype(np.float64)
    W = T[:, :, :3] @ Q.T
    t = T[:, :, 3] - np.einsum("vij,j->vi", W, s)
    poses = np.concatenate([W, t[:, :, None]], axis=2)
    B = (_A @ Q @ _A.T) @ scene.B_dir.astype(np.float64)
    f = lambda a: np.ascontiguousarray(a.astype(np.float32))
    sc2 = dataclasses.replace(scene, means=f(means), quats=f(quats), B_dir=f(B))
    return sc2, dataclasses.replace(views, world_to_cam=f(poses))


@pytest.mark.parametrize("with_dir", [False, True])
def test_joint_rigid_motion_invariance(with_dir):
    sc = syn.uniform_cloud(400, seed=7, dir_frac=0.3 if with_dir else 0.0, dir_std=1.0)
    R0 = Rotation.from_euler("zyx", [10, -20, 5], degrees=True).as_matrix()
    views = _views([_pose(R0, [0.1, -0.05, 2.0]), _pose(np.eye(3), [0.0, 0.0, 2.2])], 4.0,
                   1 / 8, 40, 56)
    st = syn.Settings(near_plane=0.2)
    Q = Rotation.from_euler("xyz", [33, -71, 140], degrees=True).as_matrix()
    s = np.array([0.25, -0.5, 1.0])
    sc2, v2 = _move(sc, views, Q, s)
    # the moved inputs are float32-rounded: compare against the unmoved render
    # of the same float32 geometry by moving back and forth in float64 only once
    a = oracle.render(sc, views, st)
    b = oracle.render(sc2, v2, st)
    clean = (a["n_flagged"] == 0) & (b["n_flagged"] == 0)
    assert clean.mean() > 0.95
    assert np.abs(a["image"] - b["image"])[clean].max() < 2e-5
    assert a["image"].max() > 0.2


# ---------------------------------------------------------------------------
# Eq. 3 special cases
# ---------------------------------------------------------------------------

def _sigmoid(x):
    return 1 / (1 + np.exp(-x))


def test_all_isotropic_reduces_to_shared_basis_model():
    # X-Gaussian's c = sigmoid(b . f) (Sec. 3.1) is DDGS with every Gaussian isotropic
    sc = syn.uniform_cloud(50, seed=1, dir_frac=0.0)
    views = _views(_pose(np.eye(3), [0, 0, 2.0]), 4.0, 1 / 8, 8, 8)
    P = oracle.project64(sc, views, syn.Settings(near_plane=0.2))
    ref = _sigmoid(sc.feat.astype(np.float64) @ sc.b_iso.astype(np.float64))
    assert np.abs(P[0, :, 6] - ref).max() < 1e-15


def test_zero_direction_basis_gives_half():
    sc = syn.uniform_cloud(50, seed=2, dir_frac=1.0)
    sc = dataclasses.replace(sc, B_dir=np.zeros_like(sc.B_dir))
    views = _views(_pose(np.eye(3), [0, 0, 2.0]), 4.0, 1 / 8, 8, 8)
    P = oracle.project64(sc, views, syn.Settings(near_plane=0.2))
    assert np.all(P[0, :, 6] == 0.5)


def test_degree_one_radiosity_is_odd_in_direction():
    # a Gaussian at the isocenter seen from opposite sides: d -> -d, and
    # sigmoid(Y_1(-d) . B f) = 1 - sigmoid(Y_1(d) . B f)
    rng = np.random.default_rng(0)
    n = 20
    feat = rng.normal(0, 1, (n, 8))
    sc = _scene(np.zeros((n, 3)), np.full((n, 3), -3.0), np.tile([1.0, 0, 0, 0], (n, 1)),
                np.zeros(n), feat, 0, B_dir=rng.normal(0, 1, (3, 8)))
    R = Rotation.from_euler("zyx", [20, 30, -40], degrees=True).as_matrix()
    # rotate the world by pi about an axis orthogonal to the source position S:
    # the new pose W Q^T has its source at Q S = -S
    S = -R.T @ np.array([0, 0, 3.0])
    ax = np.cross(S, [0.3, -0.4, 0.5])
    Q = Rotation.from_rotvec(math.pi * ax / np.linalg.norm(ax)).as_matrix()
    Rb = R @ Q.T
    views = _views([_pose(R, [0, 0, 3.0]), _pose(Rb, [0, 0, 3.0])], 6.0, 0.1, 4, 4)
    P = oracle.project64(sc, views, syn.Settings(near_plane=0.3))
    assert np.abs(P[0, :, 6] + P[1, :, 6] - 1.0).max() < 1e-12
    assert np.abs(P[0, :, 6] - 0.5).max() > 0.1


def test_degree_one_harmonics_are_orthonormal():
    # recover Y_m(d) = logit(c) / beta with B f = beta e_m, on a sphere lattice
    m_pts = 2000
    k = np.arange(m_pts) + 0.5
    zz = 1 - 2 * k / m_pts
    ph = math.pi * (1 + 5 ** 0.5) * k
    d = np.stack([np.sqrt(1 - zz ** 2) * np.cos(ph), np.sqrt(1 - zz ** 2) * np.sin(ph), zz], 1)
    beta = 0.5
    Y = np.zeros((m_pts, 3))
    for m in range(3):
        B = np.zeros((3, 8))
        B[m, 0] = beta
        feat = np.zeros((1, 8))
        feat[0, 0] = 1.0
        sc = _scene(np.zeros((1, 3)), np.full((1, 3), -3.0), [[1.0, 0, 0, 0]], [0.0], feat, 0,
                    B_dir=B)
        poses = []
        for dv in d:
            # camera whose source sits at -3 d: third row of R is d
            z = dv
            x = np.cross([0.3, 0.5, 0.8], z)
            x /= np.linalg.norm(x)
            y = np.cross(z, x)
            poses.append(_pose(np.stack([x, y, z]), [0, 0, 3.0]))
        views = _views(poses, 6.0, 0.1, 2, 2)
        P = oracle.project64(sc, views, syn.Settings(near_plane=0.3))
        c = P[:, 0, 6]
        Y[:, m] = np.log(c / (1 - c)) / beta
    gram = 4 * math.pi * (Y.T @ Y) / m_pts
    assert np.abs(gram - np.eye(3)).max() < 5e-3, gram


def test_k_L_and_parameter_count_fixtures_are_consistent():
    g = json.load(open(os.path.join(GOLDEN, "k_L.json")))
    for L, kl in g["k_L"].items():
        assert int(L) * (int(L) + 2) == kl
    p = json.load(open(os.path.join(GOLDEN, "parameter_count.json")))
    k, L = p["k"], p["L"]
    assert 3 + 4 + 3 + 1 + k == p["floats_per_gaussian"]
    assert k + L * (L + 2) * k == p["basis_floats"]
    assert p["n_gaussians"] * p["floats_per_gaussian"] + p["basis_floats"] == p["total_floats"]


def test_joint_rasterization_attenuates_occluded_set():
    # Appendix A.2: a near-opaque isotropic Gaussian in front of a
    # direction-dependent one suppresses it by (1 - sigma_iso)
    means = np.array([[0, 0, -0.3], [0, 0, 0.3]])
    feat = np.zeros((2, 8))
    feat[0, 0] = 1.0
    feat[1, 1] = 2.0
    B = np.zeros((3, 8))
    B[1, 1] = 1.0  # Y_1^0 = C1 d_z picks the beam direction
    b = np.zeros(8)
    b[0] = 1.0
    a_iso, a_dir = 0.98, 0.6
    sc = _scene(means, np.full((2, 3), math.log(0.05)), np.tile([1.0, 0, 0, 0], (2, 1)),
                syn.logit(np.array([a_iso, a_dir])), feat, 1, b_iso=b, B_dir=B)
    views = _views(_pose(np.eye(3), [0.0, 0.0, 2.0]), 4.0, 0.05, 3, 3)
    st = syn.Settings(near_plane=0.2, dilation=0.0)
    joint = oracle.render(sc, views, st)["image"][0, 1, 1]
    iso_only = dataclasses.replace(sc, means=sc.means[:1], log_scales=sc.log_scales[:1],
                                   quats=sc.quats[:1], opacity_logits=sc.opacity_logits[:1],
                                   feat=sc.feat[:1], n_iso=1)
    dir_only = dataclasses.replace(sc, means=sc.means[1:], log_scales=sc.log_scales[1:],
                                   quats=sc.quats[1:], opacity_logits=sc.opacity_logits[1:],
                                   feat=sc.feat[1:], n_iso=0)
    ci = oracle.render(iso_only, views, st)["image"][0, 1, 1]
    cd = oracle.render(dir_only, views, st)["image"][0, 1, 1]
    a32 = _sigmoid(sc.opacity_logits.astype(np.float64))
    assert abs(joint - (ci + cd * (1 - a32[0]))) < 1e-12
    assert cd > 0.3 and (ci + cd) - joint > 0.25


# ---------------------------------------------------------------------------
# Analytic gradient against central finite differences (FP64)
# ---------------------------------------------------------------------------

def _fd_scene():
    sc = syn.uniform_cloud(6, seed=21, extent=0.5, log_scale_range=(-2.2, -1.4),
                           alpha_range=(0.2, 0.7), dir_frac=0.5, dir_std=1.0)
    R1 = Rotation.from_euler("zyx", [15, -10, 25], degrees=True).as_matrix()
    views = _views([_pose(np.eye(3), [0.02, -0.03, 2.0]), _pose(R1, [0.1, 0.05, 2.3])], 4.0,
                   0.2, 20, 24)
    st = syn.Settings(near_plane=0.2, t_min=1e-3)
    return sc, views, st


def test_fd_scene_has_no_near_threshold_decision():
    sc, views, st = _fd_scene()
    r = oracle.render(sc, views, st)
    assert r["flags"].max() == 0
    assert r["n_contrib"].max() >= 3


def _loss(sc, views, st, w, depth32):
    return float((oracle.render(sc, views, st, depth32=depth32)["image"] * w).sum())


def test_analytic_gradient_matches_central_differences():
    sc, views, st = _fd_scene()
    depth32 = oracle.project32(sc, views, st)["depth"]  # order fixed: depths well apart
    rng = np.random.default_rng(3)
    w = rng.uniform(-1, 1, (views.n_views, views.height, views.width))
    g = oracle.render_backward(sc, views, st, w, depth32=depth32)
    # perturb float64 copies of the inputs (the FP64 renderer reads them exactly)
    sc64 = dataclasses.replace(sc, **{f: getattr(sc, f).astype(np.float64) for f in
                                      ("means", "log_scales", "quats", "opacity_logits",
                                       "feat", "b_iso", "B_dir")})
    v64 = dataclasses.replace(views, world_to_cam=views.world_to_cam.astype(np.float64))
    checked = 0
    groups = [(n, getattr(sc64, n), n) for n in ("means", "log_scales", "quats",
                                                  "opacity_logits", "feat", "b_iso", "B_dir")]
    groups.append(("pose", v64.world_to_cam, "pose"))
    for name, arr, gname in groups:
        G = g[gname].reshape(-1)
        scale = np.abs(G).max()
        assert scale > 0, name
        for idx in range(arr.size):
            x0 = arr.reshape(-1)[idx]
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2.reshape(-1)[idx] = x0 + sgn * h
                if name == "pose":
                    vals.append(_loss(sc64, dataclasses.replace(v64, world_to_cam=a2), st, w,
                                      depth32))
                else:
                    vals.append(_loss(dataclasses.replace(sc64, **{name: a2}), v64, st, w,
                                      depth32))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - G[idx]) <= 1e-6 * scale + 1e-9, (name, idx, fd, G[idx])
            checked += 1
    assert checked > 150


def test_count_inside_matches_brute_force():
    sc = syn.uniform_cloud(60, seed=9)
    views = _views(_pose(np.eye(3), [0.0, 0.0, 2.0]), 4.0, 0.25, 16, 20)
    st = syn.Settings(near_plane=0.2)
    n_in = oracle.count_inside(sc, views, st)
    P = oracle.project64(sc, views, st)[0]
    jj, ii = np.meshgrid(np.arange(20) + 0.5, np.arange(16) + 0.5)
    ref = np.zeros((16, 20), np.int64)
    for u, v, a, b, c, _, _, _, valid in P:
        if valid:
            dx, dy = u - jj, v - ii
            ref += (a * dx * dx + 2 * b * dx * dy + c * dy * dy) <= st.q_max
    assert np.array_equal(n_in[0], ref) and ref.sum() > 50


# ---------------------------------------------------------------------------
# Degrees L = 2, 3 of the direction decomposition (Eq. 3, Table 2)
# ---------------------------------------------------------------------------

def _lattice(m_pts):
    k = np.arange(m_pts) + 0.5
    zz = 1 - 2 * k / m_pts
    ph = math.pi * (1 + 5 ** 0.5) * k
    return np.stack([np.sqrt(1 - zz ** 2) * np.cos(ph), np.sqrt(1 - zz ** 2) * np.sin(ph), zz], 1)


def _sh_values(dirs, L, return_dirs=False):
    """Y_j(d) of the oracle for every direction, recovered from the radiosity
    sigmoid(beta Y_j) of one direction-dependent Gaussian at the isocenter.
    The cameras are float32, so the directions the oracle sees are returned too."""
    kl = L * (L + 2)
    beta = 0.5
    Y = np.zeros((dirs.shape[0], kl))
    poses = []
    for dv in dirs:
        x = np.cross([0.3, 0.5, 0.8], dv)
        x /= np.linalg.norm(x)
        poses.append(_pose(np.stack([x, np.cross(dv, x), dv]), [0, 0, 3.0]))
    views = _views(poses, 6.0, 0.1, 2, 2)
    for j in range(kl):
        B = np.zeros((kl, 8))
        B[j, 0] = beta
        feat = np.zeros((1, 8))
        feat[0, 0] = 1.0
        sc = _scene(np.zeros((1, 3)), np.full((1, 3), -3.0), [[1.0, 0, 0, 0]], [0.0], feat, 0,
                    B_dir=B)
        c = oracle.project64(sc, views, syn.Settings(near_plane=0.3))[:, 0, 6]
        Y[:, j] = np.log(c / (1 - c)) / beta
    if return_dirs:
        T = views.world_to_cam.astype(np.float64)
        d = np.einsum("vji,vj->vi", T[:, :, :3], T[:, :, 3])  # mu - S = W^T t at mu = 0
        return Y, d / np.linalg.norm(d, axis=1, keepdims=True)
    return Y


def test_harmonics_to_degree_three_are_orthonormal_with_closed_form_zonals():
    dirs = _lattice(6000)
    Y, deff = _sh_values(dirs, 3, return_dirs=True)
    gram = 4 * math.pi * (Y.T @ Y) / dirs.shape[0]
    assert np.abs(gram - np.eye(15)).max() < 3e-3, np.abs(gram - np.eye(15)).max()
    z = deff[:, 2]
    # m = 0 members: sqrt((2l+1)/4pi) P_l(z)
    assert np.allclose(Y[:, 1], math.sqrt(3 / (4 * math.pi)) * z, atol=1e-9)
    assert np.allclose(Y[:, 5], math.sqrt(5 / (16 * math.pi)) * (3 * z ** 2 - 1), atol=1e-9)
    assert np.allclose(Y[:, 11], math.sqrt(7 / (16 * math.pi)) * (5 * z ** 3 - 3 * z), atol=1e-9)


def test_harmonic_degrees_have_parity_and_are_closed_under_rotation():
    rng = np.random.default_rng(4)
    dirs = _lattice(300)
    Y = _sh_values(dirs, 3)
    Yn = _sh_values(-dirs, 3)
    for l in (1, 2, 3):
        sl = slice(l * l - 1, l * l - 1 + 2 * l + 1)
        assert np.allclose(Yn[:, sl], (-1) ** l * Y[:, sl], atol=1e-6)
    Q = Rotation.random(random_state=rng).as_matrix()
    YQ = _sh_values(dirs @ Q.T, 3)
    for l in (1, 2, 3):
        sl = slice(l * l - 1, l * l - 1 + 2 * l + 1)
        D, res, *_ = np.linalg.lstsq(Y[:, sl], YQ[:, sl], rcond=None)
        # the degree-l span is closed under rotation (up to the float32 cameras'
        # ~1e-7 direction error) and the map is orthogonal
        assert np.abs(Y[:, sl] @ D - YQ[:, sl]).max() < 1e-6
        assert np.allclose(D.T @ D, np.eye(2 * l + 1), atol=1e-6)


def test_analytic_gradient_matches_central_differences_degree_three():
    R1 = Rotation.from_euler("zyx", [25, -15, 10], degrees=True).as_matrix()
    views = _views([_pose(np.eye(3), [0.02, -0.03, 2.0]), _pose(R1, [0.1, 0.05, 2.3])], 4.0, 0.2,
                   18, 22)
    st = syn.Settings(near_plane=0.2, t_min=1e-3)
    rng = np.random.default_rng(1)
    for seed in range(23, 80):  # the first scene with no decision near a cutoff
        sc = syn.uniform_cloud(5, seed=seed, extent=0.5, log_scale_range=(-2.2, -1.4),
                               alpha_range=(0.2, 0.7), dir_frac=0.6, dir_std=1.0, k=4)
        sc = dataclasses.replace(sc, B_dir=(rng.standard_normal((15, 4)) / 2).astype(np.float32))
        if oracle.render(sc, views, st)["flags"].max() == 0:
            break
    assert oracle.render(sc, views, st)["flags"].max() == 0
    depth32 = oracle.project32(sc, views, st)["depth"]
    w = rng.uniform(-1, 1, (2, 18, 22))
    g = oracle.render_backward(sc, views, st, w, depth32=depth32)
    sc64 = dataclasses.replace(sc, **{f: getattr(sc, f).astype(np.float64) for f in
                                      ("means", "feat", "B_dir")})
    v64 = dataclasses.replace(views, world_to_cam=views.world_to_cam.astype(np.float64))
    for name, arr in (("means", sc64.means), ("feat", sc64.feat), ("B_dir", sc64.B_dir),
                      ("pose", v64.world_to_cam)):
        G = g[name].reshape(-1)
        scale = np.abs(G).max()
        for idx in range(arr.size):
            x0 = arr.reshape(-1)[idx]
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2.reshape(-1)[idx] = x0 + sgn * h
                if name == "pose":
                    vals.append(_loss(sc64, dataclasses.replace(v64, world_to_cam=a2), st, w, depth32))
                else:
                    vals.append(_loss(dataclasses.replace(sc64, **{name: a2}), v64, st, w, depth32))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - G[idx]) <= 1e-6 * scale + 1e-9, (name, idx, fd, G[idx])


# ---------------------------------------------------------------------------
# Eq. 3 variants: direct-entangled radiosity (Table 3) and per-pixel ray angles
# ---------------------------------------------------------------------------

def _logit(c):
    return np.log(c) - np.log1p(-c)


def test_entangled_logit_is_sum_of_the_two_terms():
    # co-located terms (direct-entangled, Table 3): the logit of c is b_iso . f
    # + Y(d) . B_dir f, i.e. the isotropic-only logit plus the direction-only one
    sc = syn.uniform_cloud(40, seed=31, dir_frac=0.5, dir_std=1.0)
    R = Rotation.from_euler("zyx", [30, -20, 10], degrees=True).as_matrix()
    views = _views([_pose(np.eye(3), [0, 0, 2.0]), _pose(R, [0.1, -0.2, 2.5])], 4.0, 1 / 8, 8, 8)
    st = syn.Settings(near_plane=0.2)
    ent = oracle.project64(dataclasses.replace(sc, entangled=True), views, st)[..., 6]
    iso = oracle.project64(dataclasses.replace(sc, n_iso=sc.n), views, st)[..., 6]
    dr = oracle.project64(dataclasses.replace(sc, n_iso=0), views, st)[..., 6]
    assert np.abs(_logit(ent) - (_logit(iso) + _logit(dr))).max() < 1e-9
    assert np.abs(ent - iso).max() > 1e-3 and np.abs(ent - dr).max() > 1e-3


def test_entangled_reduces_to_either_term_alone():
    sc = syn.uniform_cloud(300, seed=32, dir_frac=0.3, dir_std=1.0)
    views = _views(_pose(np.eye(3), [0, 0, 2.0]), 4.0, 1 / 8, 40, 40)
    st = syn.Settings(near_plane=0.2)
    no_dir = dataclasses.replace(sc, B_dir=np.zeros_like(sc.B_dir))
    a = oracle.render(dataclasses.replace(no_dir, entangled=True), views, st)["image"]
    b = oracle.render(dataclasses.replace(no_dir, n_iso=sc.n), views, st)["image"]
    assert np.array_equal(a, b)
    no_iso = dataclasses.replace(sc, b_iso=np.zeros_like(sc.b_iso))
    a = oracle.render(dataclasses.replace(no_iso, entangled=True), views, st)["image"]
    b = oracle.render(dataclasses.replace(no_iso, n_iso=0), views, st)["image"]
    assert np.abs(a - b).max() < 1e-15


def _centred_views(sc, st, poses, sdd, pitch, H, W):
    """Views whose principal points are shifted so that Gaussian 0's mean
    projects exactly onto the centre of pixel (H//2, W//2)."""
    # float64 poses: exactly orthonormal, so -W^T t is the source position
    P64 = np.stack([syn.pose_matrix(R, t) for R, t in poses]).astype(np.float64)
    views = syn.Views(P64, syn.detector(len(poses), sdd, pitch).astype(np.float64), H, W)
    P = oracle.project64(sc, views, st)
    det = views.detector.astype(np.float64).copy()
    det[:, 3] += (W // 2 + 0.5) - P[:, 0, 0]
    det[:, 4] += (H // 2 + 0.5) - P[:, 0, 1]
    return dataclasses.replace(views, detector=det)


def test_per_pixel_direction_equals_mean_direction_on_the_ray_through_the_mean():
    # at the pixel whose ray passes through a Gaussian's mean, the pixel ray's
    # direction and the source-to-mean direction coincide, so the two readings
    # of the ray angles give the same colour there and differ elsewhere
    rng = np.random.default_rng(5)
    n = 1
    sc = _scene(rng.uniform(-0.2, 0.2, (n, 3)), np.full((n, 3), -1.6), [[0.9, 0.1, -0.3, 0.2]],
                [0.4], rng.normal(0, 1, (n, 8)), 0, B_dir=rng.normal(0, 1, (3, 8)))
    st = syn.Settings(near_plane=0.2)
    Rs = [Rotation.from_euler("zyx", a, degrees=True).as_matrix()
          for a in ([0, 0, 0], [35, -20, 15], [-50, 40, 5])]
    views = _centred_views(sc, st, [(R, np.array([0.05, -0.1, 2.0])) for R in Rs], 4.0, 0.05, 31, 31)
    d32 = np.ones((3, 1), np.float32)  # one Gaussian: the depth order is trivial
    pg = oracle.render(sc, views, st, depth32=d32)["image"]
    pp = oracle.render(dataclasses.replace(sc, per_pixel=True), views, st, depth32=d32)["image"]
    assert np.abs(pp[:, 15, 15] - pg[:, 15, 15]).max() < 1e-12
    assert pg[:, 15, 15].min() > 0.05
    inside = pg > 1e-3
    assert np.abs(pp - pg)[inside].max() > 1e-4


def test_per_pixel_colour_follows_the_source_to_detector_geometry():
    # C(p) / sigma(p) at each pixel is sigmoid(Y_1(d_p) . B f), with d_p from
    # the source S = -R^T t to the pixel's point on the detector plane
    rng = np.random.default_rng(6)
    sc = _scene([[0.05, -0.02, 0.1]], [[-1.5, -1.7, -1.6]], [[0.8, -0.2, 0.4, 0.1]], [0.0],
                rng.normal(0, 1, (1, 8)), 0, B_dir=rng.normal(0, 1, (3, 8)))
    R = Rotation.from_euler("zyx", [20, 25, -30], degrees=True).as_matrix()
    t = np.array([0.1, 0.05, 2.2])
    H = W = 25
    views = _views(_pose(R, t), 4.4, 0.06, H, W, off=(0.7, -1.3))
    st = syn.Settings(near_plane=0.2)
    pg = oracle.render(sc, views, st)
    pp = oracle.render(dataclasses.replace(sc, per_pixel=True), views, st)["image"][0]
    c_mean = oracle.project64(sc, views, st)[0, 0, 6]
    sigma = pg["image"][0] / c_mean
    Rf, tf = views.world_to_cam[0, :, :3].astype(np.float64), views.world_to_cam[0, :, 3].astype(np.float64)
    S = -Rf.T @ tf
    h = sc.B_dir.astype(np.float64) @ sc.feat[0].astype(np.float64)
    det = views.detector[0].astype(np.float64)
    ok = pg["n_contrib"][0] > 0
    assert ok.sum() > 20
    for i, j in zip(*np.nonzero(ok)):
        Pc = np.array([(j + 0.5 - (W / 2 + det[3])) * det[1], (i + 0.5 - (H / 2 + det[4])) * det[2],
                       det[0]])
        d = Rf.T @ (Pc - tf) - S
        d /= np.linalg.norm(d)
        Y1 = math.sqrt(3 / (4 * math.pi)) * np.array([-d[1], d[2], -d[0]])
        assert abs(pp[i, j] - sigma[i, j] * _sigmoid(Y1 @ h)) < 1e-12


def _fd_check(sc, views, st, names, seed=3):
    depth32 = oracle.project32(sc, views, st)["depth"]
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1, 1, (views.n_views, views.height, views.width))
    g = oracle.render_backward(sc, views, st, w, depth32=depth32)
    sc64 = dataclasses.replace(sc, **{f: getattr(sc, f).astype(np.float64) for f in
                                      ("means", "log_scales", "quats", "opacity_logits",
                                       "feat", "b_iso", "B_dir")})
    v64 = dataclasses.replace(views, world_to_cam=views.world_to_cam.astype(np.float64))
    checked = 0
    for name in names:
        arr = v64.world_to_cam if name == "pose" else getattr(sc64, name)
        G = g[name].reshape(-1)
        scale = np.abs(G).max()
        assert scale > 0, name
        for idx in range(arr.size):
            x0 = arr.reshape(-1)[idx]
            hh = 1e-6 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2.reshape(-1)[idx] = x0 + sgn * hh
                if name == "pose":
                    vals.append(_loss(sc64, dataclasses.replace(v64, world_to_cam=a2), st, w, depth32))
                else:
                    vals.append(_loss(dataclasses.replace(sc64, **{name: a2}), v64, st, w, depth32))
            fd = (vals[0] - vals[1]) / (2 * hh)
            assert abs(fd - G[idx]) <= 1e-6 * scale + 1e-9, (name, idx, fd, G[idx])
            checked += 1
    return checked


@pytest.mark.parametrize("entangled,per_pixel", [(True, False), (False, True), (True, True)])
def test_variant_gradients_match_central_differences(entangled, per_pixel):
    sc, views, st = _fd_scene()
    sc = dataclasses.replace(sc, entangled=entangled, per_pixel=per_pixel)
    assert oracle.render(sc, views, st)["flags"].max() == 0
    n = _fd_check(sc, views, st, ("means", "feat", "b_iso", "B_dir", "opacity_logits", "pose"))
    assert n > 100
