"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Sizes are chosen so the oracle finishes in seconds while spanning several
tiles and ragged tile edges; the full-size workloads are checked on sampled
pixels. Tolerances are in tests/_parity.py.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn
from _parity import check_image, compare_binning, compare_grads, gradient_weights, last_ids

pytestmark = pytest.mark.gpu

GRAD_NAMES = ["means", "log_scales", "quats", "opacity_logits", "feat", "b_iso", "B_dir", "pose"]


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


def _views(poses, sdd, pitch, H, W):
    poses = np.ascontiguousarray(np.asarray(poses, np.float32).reshape(-1, 3, 4))
    return syn.Views(poses, syn.detector(poses.shape[0], sdd, pitch), H, W)


def _two_views(H, W, pitch=8.0 / 96):
    return _views([syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])),
                   syn.pose_matrix(syn.rot_y(0.5) @ syn.rot_x(-0.2), np.array([0.05, -0.1, 2.3]))],
                  4.0, pitch, H, W)


def _run(scene, views, st, ws, bf16=None, depth=None):
    cloud = B.cloud_from_arrays(scene, feat_dir_bf16=bf16)
    gv = B.views_from_arrays(views)
    cfg = B.config_from_settings(st) if depth is None else B.config_from_settings(st, batch_depth=depth)
    img, tf, nl = B.render(cloud, gv, cfg, ws)
    torch.cuda.synchronize()
    return cloud, gv, cfg, img, tf, nl


def _bins(ws, scene, views, st):
    t = st.tile
    tiles = views.n_views * (-(-views.width // t)) * (-(-views.height // t))
    return B.debug_binning(ws, views.n_views, scene.n, tiles)


def _crowded(n, extent, seed, z_levels=None):
    """n Gaussians packed into a small cube at the isocentre (long tile lists);
    with z_levels the means take only those depths (many exact depth ties)."""
    sc = syn.uniform_cloud(n, seed=seed, extent=extent, log_scale_range=(-5.0, -4.0))
    if z_levels is not None:
        rng = np.random.default_rng(seed + 1)
        means = sc.means.copy()
        means[:, 2] = np.asarray(z_levels, np.float32)[rng.integers(0, len(z_levels), n)]
        sc = dataclasses.replace(sc, means=means)
    return sc


def _plane(n, seed):
    """Means on the plane z = 0 facing the first view: every depth of that view
    is the same, so its lists are ordered by Gaussian index alone."""
    sc = syn.uniform_cloud(n, seed=seed)
    means = sc.means.copy()
    means[:, 2] = 0.0
    return dataclasses.replace(sc, means=means)


CASES = {
    "plain_4096_128px": lambda: syn.plain_forward_workload(),
    # one tile of each view holds 20k pairs: chunks sorted by blocks, then merged
    "crowded_long_lists": lambda: (_crowded(20000, 0.05, 11, z_levels=(-0.01, 0.0, 0.01)),
                                   _two_views(48, 48, 8.0 / 48), syn.Settings(near_plane=0.2, tile=16)),
    # lists of a few hundred to a few thousand pairs around the centre
    "crowded_block_lists": lambda: (_crowded(12000, 0.3, 12), _two_views(64, 64, 8.0 / 64),
                                    syn.Settings(near_plane=0.2, tile=8)),
    "equal_depths": lambda: (_plane(3000, 13), _two_views(64, 64, 8.0 / 64),
                             syn.Settings(near_plane=0.2, tile=16)),
    # footprints of up to the whole view: binning rounds too large to stage
    "large_footprints": lambda: (syn.uniform_cloud(4000, seed=14, log_scale_range=(-1.5, -0.5)),
                                 _two_views(64, 64, 8.0 / 64), syn.Settings(near_plane=0.2, tile=8)),
    "ragged_100x75_2views": lambda: (syn.uniform_cloud(2000, seed=5), _two_views(75, 100),
                                     syn.Settings(near_plane=0.2)),
    "tile8": lambda: (syn.uniform_cloud(1500, seed=6), _two_views(41, 57, 8.0 / 50),
                      syn.Settings(near_plane=0.2, tile=8)),
    "tile32": lambda: (syn.uniform_cloud(1500, seed=7), _two_views(70, 90, 8.0 / 80),
                       syn.Settings(near_plane=0.2, tile=32)),
    "strong_dir": lambda: (syn.uniform_cloud(1200, seed=8, dir_frac=0.5, dir_std=1.0),
                           _two_views(48, 64, 8.0 / 60), syn.Settings(near_plane=0.2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_binning_is_bit_exact(case, ws):
    scene, views, st = CASES[case]()
    _run(scene, views, st, ws)
    gpu = _bins(ws, scene, views, st)
    ref = oracle.bin32(scene, views, st)
    compare_binning(gpu, ref)


@pytest.mark.parametrize("case", sorted(CASES))
def test_image_matches_oracle(case, ws):
    scene, views, st = CASES[case]()
    _, _, _, img, tf, nl = _run(scene, views, st, ws)
    bins = _bins(ws, scene, views, st)
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids,
                      depth32=bins_depth(scene, views, st))
    assert rep["range"] > 0.1
    assert rep["unresolved_frac"] <= 1e-3


def bins_depth(scene, views, st):
    return oracle.project32(scene, views, st)["depth"]


def _resolved_weights(scene, views, st, ws, img, tf, nl, seed):
    """Image check of the last render, then the loss weights of a gradient
    check: every pixel resolved to the oracle outcome the GPU took (the oracle
    differentiates it along that outcome), at most 1e-3 of a view left out."""
    bins = _bins(ws, scene, views, st)
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    w, fm = gradient_weights(rep, seed)
    return rep, w, fm


@pytest.mark.parametrize("case", ["plain_4096_128px", "ragged_100x75_2views", "strong_dir",
                                  "tile8", "tile32"])
def test_gradients_match_oracle(case, ws):
    scene, views, st = CASES[case]()
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    _, w, fm = _resolved_weights(scene, views, st, ws, img, tf, nl, 0)
    dL = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    g = B.render_backward(cloud, gv, cfg, ws, dL, tf, nl)
    torch.cuda.synchronize()
    gr = oracle.render_backward(scene, views, st, w, flip_masks=fm)
    gpu = {k: v.cpu().numpy() for k, v in g.items()}
    gpu["feat"] = np.concatenate([gpu.pop("feat_iso"), gpu.pop("feat_dir")])
    gpu["pose"] = gpu.pop("world_to_cam")
    compare_grads(gpu, gr, GRAD_NAMES)


def test_bf16_direction_features(ws):
    ph = syn.make_phantom(48, seed=2, fov=96.0)
    scene = syn.gaussians_from_phantom(ph, 3000, seed=2, bf16_dir=True)
    views = syn.Views(syn.orbit_poses(2, 300.0), syn.detector(2, 375.0, 96.0 / 64), 64, 64)
    st = syn.Settings(near_plane=30.0)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws, bf16=True)
    assert cloud.feat_dir.dtype == torch.bfloat16
    bins = _bins(ws, scene, views, st)
    compare_binning(bins, oracle.bin32(scene, views, st))
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    w, fm = gradient_weights(rep, 1)
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl)
    gr = oracle.render_backward(scene, views, st, w, flip_masks=fm)
    gpu = {k: v.float().cpu().numpy() for k, v in g.items()}
    gpu["feat"] = np.concatenate([gpu.pop("feat_iso"), gpu.pop("feat_dir")])
    gpu["pose"] = gpu.pop("world_to_cam")
    compare_grads(gpu, gr, GRAD_NAMES)


def test_empty_and_degenerate_inputs(ws):
    # no Gaussians
    scene = syn.uniform_cloud(0, seed=0)
    views = _two_views(20, 30)
    st = syn.Settings(near_plane=0.2)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    assert float(img.abs().max()) == 0.0 and float(tf.min()) == 1.0 and int(nl.max()) == 0
    g = B.render_backward(cloud, gv, cfg, ws, torch.ones_like(img), tf, nl,
                          want=["world_to_cam", "b_iso", "B_dir"])
    assert float(g["world_to_cam"].abs().max()) == 0.0
    # every Gaussian behind the near plane or beyond the detector
    scene = syn.uniform_cloud(300, seed=1)
    scene.means[:, 2] = np.where(np.arange(300) % 2 == 0, -1.95, 2.5).astype(np.float32)
    view1 = _views(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])), 4.0, 8.0 / 30, 20, 30)
    cloud, gv, cfg, img, tf, nl = _run(scene, view1, st, ws)
    assert float(img.abs().max()) == 0.0 and ws.pairs() == 0
    # all isotropic / all direction-dependent
    for frac in (0.0, 1.0):
        scene = syn.uniform_cloud(400, seed=2, dir_frac=frac)
        views1 = _two_views(33, 47, 8.0 / 40)
        _, _, _, img, tf, nl = _run(scene, views1, st, ws)
        bins = _bins(ws, scene, views1, st)
        compare_binning(bins, oracle.bin32(scene, views1, st))
        ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views1, st.tile)
        check_image(scene, views1, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    # a single pixel detector, a single Gaussian
    scene = syn.uniform_cloud(1, seed=3, log_scale_range=(-1.0, -0.9))
    scene.means[:] = 0
    views1 = _views(syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])), 4.0, 0.5, 1, 1)
    _, _, _, img, tf, nl = _run(scene, views1, st, ws)
    ref = oracle.render(scene, views1, st)
    assert abs(float(img[0, 0, 0]) - ref["image"][0, 0, 0]) < 1e-6
    assert int(nl[0, 0, 0]) == 1


def test_autograd_function_matches_direct_backward(ws):
    scene, views, st = CASES["ragged_100x75_2views"]()
    cloud = B.cloud_from_arrays(scene)
    gv = B.views_from_arrays(views)
    cfg = B.config_from_settings(st)
    params = [cloud.means, cloud.log_scales, cloud.quats, cloud.opacity_logits, cloud.feat_iso,
              cloud.feat_dir, cloud.b_iso, cloud.B_dir, gv.world_to_cam]
    for p in params:
        p.requires_grad_(True)
    img, tf, nl = B.render_differentiable(cloud, gv, cfg, ws)
    w = torch.linspace(-1, 1, img.numel(), device="cuda").reshape(img.shape)
    (img * w).sum().backward()
    grads_auto = [p.grad.clone() for p in params]
    cloud2 = B.Cloud(*[p.detach() for p in params[:8]])
    gv2 = B.Views(gv.world_to_cam.detach(), gv.detector, gv.height, gv.width)
    img2, tf2, nl2 = B.render(cloud2, gv2, cfg, ws)
    g = B.render_backward(cloud2, gv2, cfg, ws, w, tf2, nl2)
    torch.cuda.synchronize()
    assert torch.equal(img.detach(), img2)
    names = ["means", "log_scales", "quats", "opacity_logits", "feat_iso", "feat_dir", "b_iso",
             "B_dir", "world_to_cam"]
    for ga, n in zip(grads_auto, names):
        scale = float(g[n].abs().max()) + 1e-30
        assert float((ga - g[n]).abs().max()) <= 1e-5 * scale, n


def test_gpu_fp32_gradient_agrees_with_finite_differences(ws):
    # sanity only: FP32 renders, steps large enough to be resolved in FP32,
    # cutoffs pushed out so that a step cannot flip a visible decision
    scene = syn.uniform_cloud(6, seed=21, extent=0.5, log_scale_range=(-2.2, -1.4),
                              alpha_range=(0.2, 0.7), dir_frac=0.5, dir_std=1.0)
    views = _two_views(20, 24, 0.2)
    st = syn.Settings(near_plane=0.2, t_min=1e-7, alpha_min=1e-7, q_max=30.0)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    w = torch.as_tensor(np.random.default_rng(3).uniform(-1, 1, img.shape), dtype=torch.float32,
                        device="cuda")
    g = B.render_backward(cloud, gv, cfg, ws, w, tf, nl, want=["means", "world_to_cam"])
    for name, tensor in (("means", cloud.means), ("world_to_cam", gv.world_to_cam)):
        G = g[name].reshape(-1).cpu().numpy()
        base = tensor.clone()
        fd = np.zeros_like(G)
        for idx in range(G.size):
            vals = []
            for sgn in (1, -1):
                t = base.clone().reshape(-1)
                t[idx] += sgn * 1e-3
                tensor.copy_(t.reshape(base.shape))
                im, _, _ = B.render(cloud, gv, cfg, ws)
                vals.append(float((im * w).double().sum()))
            fd[idx] = (vals[0] - vals[1]) / 2e-3
        tensor.copy_(base)
        err = np.abs(fd - G).max() / np.abs(G).max()
        assert err < 2e-2, (name, err)


def test_l1_loss_kernel(ws):
    rng = np.random.default_rng(0)
    img = torch.as_tensor(rng.uniform(0, 1, (3, 17, 23)), dtype=torch.float32, device="cuda")
    tgt = torch.as_tensor(rng.uniform(0, 1, (17, 23)), dtype=torch.float32, device="cuda")
    loss, grad = B.l1_loss(img, tgt)
    torch.cuda.synchronize()
    d = img.cpu().numpy().astype(np.float64) - tgt.cpu().numpy()[None]
    assert np.allclose(loss.cpu().numpy(), np.abs(d).mean(axis=(1, 2)), rtol=1e-5)
    assert np.array_equal(grad.cpu().numpy(), (np.sign(d) / (17 * 23)).astype(np.float32))


@pytest.mark.parametrize("direct", [False, True])
def test_capacity_overflow_is_reported_not_faulted(direct, ws):
    """A no-sync render with too small a pair capacity drops whole lists and
    reports it. direct: large footprints and a capacity of about 60 % of the
    pairs, so that the scatter takes its unstaged instance (its blocks average
    more pairs than two staging windows) and still overflows."""
    scene = syn.uniform_cloud(20000, seed=5, **({"log_scale_range": (-1.5, -0.5)} if direct else {}))
    views = _two_views(75, 100)
    st = syn.Settings(near_plane=0.2)
    m_needed = oracle.bin32(scene, views, st)["m"]
    w2 = B.Workspace()
    recs = views.n_views * scene.n
    cap = m_needed // 2 if direct else 64
    w2.reserve(recs, cap, views.n_views * 42)  # fewer pairs than needed
    granted = cap + cap // 4 + 4096  # what the workspace reserves for cap
    assert m_needed > granted
    if direct:  # 10 chunks per view, 2 views: the unstaged scatter from 204,800 pairs
        assert granted > 2 * 5120 * 20
    cloud = B.cloud_from_arrays(scene)
    gv = B.views_from_arrays(views)
    cfg = B.config_from_settings(st, no_sync=True)
    B.render(cloud, gv, cfg, w2)
    assert w2.sync_status() == 2  # DDGS_ERR_CAPACITY
    assert w2.sync_status() == 0  # cleared
    # whole lists only: the lists that fit are the first tiles' lists, exactly
    # the oracle's; every list after the first one that did not fit is empty
    ref = oracle.bin32(scene, views, st)
    got = _bins(w2, scene, views, st)
    rr, gr = ref["ranges"].reshape(-1, 2).astype(np.int64), got["ranges"].reshape(-1, 2).astype(np.int64)
    kept, has = gr[:, 1] > gr[:, 0], rr[:, 1] > rr[:, 0]
    assert kept.any() and not kept.all()
    first_drop = int(np.argmax(has & ~kept))
    assert not kept[first_drop:].any()
    for t in np.nonzero(kept)[0]:
        assert np.array_equal(got["vals"][gr[t, 0]:gr[t, 1]], ref["vals"][rr[t, 0]:rr[t, 1]])
    # the same workspace renders correctly once it is large enough
    w2.reserve(recs, m_needed, views.n_views * 42)
    img, tf, nl = B.render(cloud, gv, cfg, w2)
    assert w2.sync_status() == 0
    img_ref, _, _ = B.render(cloud, gv, B.config_from_settings(st), ws)
    torch.cuda.synchronize()
    assert torch.equal(img, img_ref)
    w2.close()


def _compare_view_lists(gpu, ref, views_gpu, tiles_per_view):
    """Tile lists of some views of a render (gpu: every view; ref: the FP32
    binning reference of those views alone, in that order): per tile the same
    range length, Gaussians and depth keys, entry for entry."""
    gr = gpu["ranges"].reshape(-1, 2).astype(np.int64)
    rr = ref["ranges"].reshape(-1, 2).astype(np.int64)
    for j, v in enumerate(views_gpu):
        g = gr[v * tiles_per_view:(v + 1) * tiles_per_view]
        r = rr[j * tiles_per_view:(j + 1) * tiles_per_view]
        assert np.array_equal(g[:, 1] - g[:, 0], r[:, 1] - r[:, 0]), f"list lengths of view {v}"
        full = g[:, 1] > g[:, 0]  # empty lists are (0, 0) on both sides
        assert np.array_equal(g[~full], r[~full]), f"empty ranges of view {v}"
        if not full.any():
            continue
        g0, g1, r0, r1 = g[full, 0].min(), g[full, 1].max(), r[full, 0].min(), r[full, 1].max()
        assert np.array_equal(g[full] - g0, r[full] - r0), f"ranges of view {v}"
        assert np.array_equal(gpu["vals"][g0:g1], ref["vals"][r0:r1]), f"lists of view {v}"
        gk, rk = gpu["keys"][g0:g1], ref["keys"][r0:r1]
        assert np.array_equal(gk & 0xffffffff, rk & 0xffffffff), f"depth keys of view {v}"
        shift = np.uint64((v - j) * tiles_per_view)
        assert np.array_equal(gk >> np.uint64(32), (rk >> np.uint64(32)) + shift), f"tiles of view {v}"


@pytest.mark.slow
def test_registration_workload_sampled_pixels(ws):
    """500k Gaussians, 64 poses, 256^2, in the launch shape the benchmark
    times (tile 8, warp-streamed rasterisers): bit-exact tile lists of two
    views against the FP32 binning reference, image and pose gradients on
    sampled pixels of those views (oracle one pixel at a time)."""
    scene, views, st = syn.registration_workload()
    st = dataclasses.replace(st, tile=8)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws, depth=32)
    bins = _bins(ws, scene, views, st)
    ref_proj = oracle.project32(scene, views, st)
    assert np.array_equal(bins["tiles_touched"].reshape(ref_proj["tiles_touched"].shape),
                          ref_proj["tiles_touched"])
    assert bins["m"] == int(ref_proj["tiles_touched"].sum())
    keys = bins["keys"]
    assert np.all(keys[1:] >= keys[:-1])
    check_views = [0, 37]
    sub = dataclasses.replace(views, world_to_cam=views.world_to_cam[check_views].copy(),
                              detector=views.detector[check_views].copy())
    # bit-exact binning of two whole views: every tile's list, entry for entry
    tpv = (views.width // 8) * (views.height // 8)
    _compare_view_lists(bins, oracle.bin32(scene, sub, st), check_views, tpv)
    pix = syn.sample_pixels(sub, n_random=768, n_rows=1, seed=4)
    sel_v = np.array(check_views)[pix[:, 0]]
    ids_all = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    gi = img.cpu().numpy()[sel_v, pix[:, 1], pix[:, 2]]
    gt = tf.cpu().numpy()[sel_v, pix[:, 1], pix[:, 2]]
    gid = ids_all[sel_v, pix[:, 1], pix[:, 2]]
    rep = check_image(scene, sub, st, gi, gt, gid, depth32=ref_proj["depth"][check_views], pix=pix)
    assert rep["range"] > 0.1
    # pose gradients of a loss on the sampled pixels only (same weights both sides)
    w = np.zeros(img.shape, np.float64)
    wv, fm = gradient_weights(rep, 9)
    w[sel_v, pix[:, 1], pix[:, 2]] = wv
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl, want=["world_to_cam"])
    gr = oracle.render_backward(scene, sub, st, wv, pix=pix, depth32=ref_proj["depth"][check_views],
                                flip_masks=fm)
    gp = g["world_to_cam"].cpu().numpy()
    compare_grads({"pose": gp[check_views]}, {"pose": gr["pose"]}, ["pose"])
    others = np.setdiff1d(np.arange(views.n_views), check_views)
    assert np.abs(gp[others]).max() == 0.0


def _sampled_check(scene, views, st, ws, check_views, n_random, seed, grads=("pose",), bf16=None,
                   depth=None):
    """Full-size render and backward on the GPU; the oracle evaluates sampled
    pixels of a few views one by one; gradients of a loss on those pixels only."""
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws, bf16=bf16, depth=depth)
    bins = _bins(ws, scene, views, st)
    ref_proj = oracle.project32(scene, views, st)
    assert np.array_equal(bins["tiles_touched"].reshape(ref_proj["tiles_touched"].shape),
                          ref_proj["tiles_touched"])
    assert bins["m"] == int(ref_proj["tiles_touched"].sum())
    assert np.all(bins["keys"][1:] >= bins["keys"][:-1])
    sub = dataclasses.replace(views, world_to_cam=views.world_to_cam[check_views].copy(),
                              detector=views.detector[check_views].copy())
    pix = syn.sample_pixels(sub, n_random=n_random, n_rows=1, seed=seed)
    sel_v = np.array(check_views)[pix[:, 0]]
    ids_all = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    gi = img.cpu().numpy()[sel_v, pix[:, 1], pix[:, 2]]
    gt = tf.cpu().numpy()[sel_v, pix[:, 1], pix[:, 2]]
    gid = ids_all[sel_v, pix[:, 1], pix[:, 2]]
    d32 = ref_proj["depth"][check_views]
    rep = check_image(scene, sub, st, gi, gt, gid, depth32=d32, pix=pix)
    assert rep["range"] > 0.05
    w = np.zeros(img.shape, np.float64)
    wv, fm = gradient_weights(rep, seed + 1)
    w[sel_v, pix[:, 1], pix[:, 2]] = wv
    want = ["world_to_cam"] + [n for n in ("means", "log_scales", "quats", "opacity_logits",
                                           "feat_iso", "feat_dir", "b_iso", "B_dir") if n in grads]
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl, want=want)
    gr = oracle.render_backward(scene, sub, st, wv, pix=pix, depth32=d32, flip_masks=fm)
    gpu = {k: v.float().cpu().numpy() for k, v in g.items()}
    gpu["pose"] = gpu.pop("world_to_cam")[check_views]
    if "feat_iso" in gpu:
        gpu["feat"] = np.concatenate([gpu.pop("feat_iso"), gpu.pop("feat_dir")])
    names = [n for n in ("means", "log_scales", "quats", "opacity_logits", "feat", "b_iso", "B_dir",
                         "pose") if n in gpu]
    compare_grads(gpu, gr, names)
    return rep


@pytest.mark.slow
@pytest.mark.parametrize("tile,depth", [(16, 256), (8, 32)])
def test_fit_workload_sampled_pixels(tile, depth, ws):
    """100k Gaussians from a 128^3 phantom, 512^2 at 0.5 mm: forward + backward
    with respect to every Gaussian parameter, the bases and the pose, in the
    block-staged launch shape and the warp-streamed one the fit benchmark
    autotunes to."""
    scene, views, st = syn.fit_workload()
    st = dataclasses.replace(st, tile=tile)
    _sampled_check(scene, views, st, ws, [0], 2048, 5, depth=depth,
                   grads=("means", "log_scales", "quats", "opacity_logits", "feat_iso", "feat_dir",
                          "b_iso", "B_dir", "pose"))


@pytest.mark.slow
@pytest.mark.parametrize("tile,depth", [(16, 256), (8, 32)])
def test_large_fit_workload_sampled_pixels(tile, depth, ws):
    """2M Gaussians from a 512^3 phantom with lesions, 8 orbit views at 1024^2,
    bf16 direction features: sampled pixels of two views, all gradients, in
    both launch shapes."""
    scene, views, st = syn.large_fit_workload()
    assert scene.feat_dir_bf16
    st = dataclasses.replace(st, tile=tile)
    _sampled_check(scene, views, st, ws, [0, 5], 640, 6, bf16=True, depth=depth,
                   grads=("means", "log_scales", "quats", "opacity_logits", "feat_iso", "feat_dir",
                          "b_iso", "B_dir", "pose"))


@pytest.mark.parametrize("k,L,bf16", [(1, 1, False), (4, 2, False), (8, 3, False), (16, 3, True),
                                      (32, 1, False), (8, 2, True)])
def test_feature_dimension_and_degree_variants(k, L, bf16, ws):
    """Tables 2 and 5 of the paper vary k (1..32) and the degree L (1, 3): the
    generic kernels against the oracle, image and every gradient."""
    scene = syn.uniform_cloud(1500, seed=50 + k + L, dir_frac=0.5, dir_std=1.0, k=k, sh_degree=L)
    if bf16:
        scene.feat[scene.n_iso:] = syn.round_to_bf16(scene.feat[scene.n_iso:])
    views = _two_views(45, 60, 8.0 / 56)
    st = syn.Settings(near_plane=0.2)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws, bf16=bf16)
    assert cloud.feat_dim == k and cloud.sh_degree == L
    bins = _bins(ws, scene, views, st)
    compare_binning(bins, oracle.bin32(scene, views, st))
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    w, fm = gradient_weights(rep, 3)
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl)
    gr = oracle.render_backward(scene, views, st, w, flip_masks=fm)
    gpu = {n: t.float().cpu().numpy() for n, t in g.items()}
    gpu["feat"] = np.concatenate([gpu.pop("feat_iso").reshape(-1, k), gpu.pop("feat_dir").reshape(-1, k)])
    gpu["pose"] = gpu.pop("world_to_cam")
    compare_grads(gpu, gr, GRAD_NAMES)


@pytest.mark.parametrize("entangled,per_pixel,tile,bf16", [
    (True, False, 16, False), (False, True, 16, False), (True, True, 16, False),
    (False, True, 8, False), (True, True, 32, True)])
def test_radiosity_variants(entangled, per_pixel, tile, bf16, ws):
    """Eq. 3 variants (direct-entangled terms, Table 3; ray angles per pixel)
    against the oracle: binning, image and every gradient, the pose included."""
    scene = syn.uniform_cloud(1500, seed=60 + tile, dir_frac=0.4, dir_std=1.0)
    scene = dataclasses.replace(scene, entangled=entangled, per_pixel=per_pixel)
    if bf16:
        scene.feat[scene.n_iso:] = syn.round_to_bf16(scene.feat[scene.n_iso:])
    views = _two_views(45, 60, 8.0 / 56)
    st = syn.Settings(near_plane=0.2, tile=tile)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws, bf16=bf16)
    assert cloud.entangled == entangled and cloud.per_pixel == per_pixel
    bins = _bins(ws, scene, views, st)
    compare_binning(bins, oracle.bin32(scene, views, st))
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    w, fm = gradient_weights(rep, 3)
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl)
    gr = oracle.render_backward(scene, views, st, w, flip_masks=fm)
    gpu = {n: t.float().cpu().numpy() for n, t in g.items()}
    gpu["feat"] = np.concatenate([gpu.pop("feat_iso").reshape(-1, 8), gpu.pop("feat_dir").reshape(-1, 8)])
    gpu["pose"] = gpu.pop("world_to_cam")
    compare_grads(gpu, gr, GRAD_NAMES)


def test_per_pixel_mode_must_match_between_forward_and_backward(ws):
    scene = syn.uniform_cloud(300, seed=70, dir_frac=0.5)
    views = _two_views(32, 32, 8.0 / 30)
    st = syn.Settings(near_plane=0.2)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    other = dataclasses.replace(cloud, per_pixel=True)
    with pytest.raises(RuntimeError):
        B.render_backward(other, gv, cfg, ws, torch.ones_like(img), tf, nl)
    # degree 3 has no per-pixel path
    sc3 = syn.uniform_cloud(300, seed=71, dir_frac=0.5, sh_degree=3)
    c3 = dataclasses.replace(B.cloud_from_arrays(sc3), per_pixel=True)
    with pytest.raises(RuntimeError):
        B.render(c3, gv, cfg, ws)


@pytest.mark.parametrize("case,per_pixel", [("ragged_100x75_2views", False), ("tile8", False),
                                            ("tile32", False), ("strong_dir", True)])
def test_warp_streamed_rasterisers(case, per_pixel, ws):
    """Staging depth 32: every warp streams its own region's list. Image and
    every gradient against the oracle."""
    scene, views, st = CASES[case]()
    scene = dataclasses.replace(scene, per_pixel=per_pixel)
    cloud = B.cloud_from_arrays(scene)
    gv = B.views_from_arrays(views)
    cfg = B.config_from_settings(st, batch_depth=32)
    img, tf, nl = B.render(cloud, gv, cfg, ws)
    torch.cuda.synchronize()
    bins = _bins(ws, scene, views, st)
    ids = last_ids(nl.cpu().numpy().view(np.uint32), bins, views, st.tile)
    rep = check_image(scene, views, st, img.cpu().numpy(), tf.cpu().numpy(), ids)
    w, fm = gradient_weights(rep, 5)
    g = B.render_backward(cloud, gv, cfg, ws, torch.as_tensor(w, dtype=torch.float32, device="cuda"),
                          tf, nl)
    gr = oracle.render_backward(scene, views, st, w, flip_masks=fm)
    gpu = {n: t.float().cpu().numpy() for n, t in g.items()}
    gpu["feat"] = np.concatenate([gpu.pop("feat_iso"), gpu.pop("feat_dir")])
    gpu["pose"] = gpu.pop("world_to_cam")
    compare_grads(gpu, gr, GRAD_NAMES)


def _banded_case(shape):
    """Views with more tiles than one binning band holds (8,192 at tile 8):
    1024 x 1024 (128 x 128 tiles: two bands of 64 tile rows) and an 8-pixel
    strip 66,000 pixels wide (one row of 8,250 tiles: two bands of columns)."""
    H, W = shape
    st = syn.Settings(near_plane=0.2, tile=8)
    views = _views([syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0]))], 4.0, 8.0 / W, H, W)
    if H > 8:
        return syn.uniform_cloud(3000, seed=21), views, st
    sc = syn.uniform_cloud(3000, seed=22, log_scale_range=(-6.0, -5.0))
    means = sc.means.copy()
    means[:, 1] *= 2e-4  # the strip is 8 pixels = 0.001 units high
    return dataclasses.replace(sc, means=means), views, st


@pytest.mark.parametrize("shape", [(1024, 1024), (8, 66000)])
def test_banded_views(shape, ws):
    scene, views, st = _banded_case(shape)
    _run(scene, views, st, ws)
    compare_binning(_bins(ws, scene, views, st), oracle.bin32(scene, views, st))
    _sampled_check(scene, views, st, ws, [0], 1024, 31, grads=("means", "opacity_logits", "pose"))


def test_backward_leaves_its_accumulators_clear(ws):
    """The backward preprocess clears every 2D-gradient record it consumes, so
    a second backward of the same render (and one after a render of another
    layout) gives the same gradients as the first."""
    scene, views, st = CASES["ragged_100x75_2views"]()
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    w = torch.as_tensor(np.random.default_rng(17).uniform(-1, 1, img.shape), dtype=torch.float32,
                        device="cuda")
    g1 = {k: v.clone() for k, v in B.render_backward(cloud, gv, cfg, ws, w, tf, nl).items()}
    g2 = B.render_backward(cloud, gv, cfg, ws, w, tf, nl)
    torch.cuda.synchronize()
    # equal up to the order of the float atomics (a record added twice would
    # be off by its whole value)
    ref = {k: v.cpu().numpy() for k, v in g1.items()}
    compare_grads({k: v.cpu().numpy() for k, v in g2.items()}, ref, list(g1), tol=1e-5,
                  zero_ok=list(g1))
    other, oviews, ost = CASES["tile8"]()
    c2, gv2, cfg2, img2, tf2, nl2 = _run(other, oviews, ost, ws)
    B.render_backward(c2, gv2, cfg2, ws, torch.ones_like(img2), tf2, nl2)
    cloud, gv, cfg, img, tf, nl = _run(scene, views, st, ws)
    g3 = B.render_backward(cloud, gv, cfg, ws, w, tf, nl)
    torch.cuda.synchronize()
    compare_grads({k: v.cpu().numpy() for k, v in g3.items()}, ref, list(g1), tol=1e-5,
                  zero_ok=list(g1))
