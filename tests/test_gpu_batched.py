"""GPU: batches of uneven requests (own cloud, bases, views and detector
sizes per request) through ddgs_render_batched / _backward.

A request rendered inside a batch must give exactly what it gives alone
(images, transmittance and list positions bit-identical: same lists, same
order), its gradients must equal the single-request ones up to the order of
atomic additions, and the images must match the oracle."""
import numpy as np
import pytest
import torch

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import synthetic as syn
from _parity import check_image, compare_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2406_02518_gb300 import build
    build.build()
    B.load()


def _requests():
    """Requests of different cloud sizes, iso/dir splits, detector sizes and
    view counts, including an empty cloud and a request with no view."""
    specs = [(900, 0.2, [(48, 40)]), (0, 0.2, [(20, 20)]), (1500, 0.5, [(33, 70), (64, 64)]),
             (400, 1.0, []), (2500, 0.0, [(17, 129)])]
    reqs = []
    for k, (n, frac, dets) in enumerate(specs):
        sc = syn.uniform_cloud(n, seed=30 + k, dir_frac=frac, dir_std=0.5)
        vs = []
        for j, (H, W) in enumerate(dets):
            P = syn.pose_matrix(syn.rot_y(0.3 * j) @ syn.rot_x(0.1 * k),
                                np.array([0.0, 0.05 * j, 2.0 + 0.1 * k]))
            vs.append(syn.Views(P[None].astype(np.float32), syn.detector(1, 4.0, 8.0 / max(H, W)), H, W))
        reqs.append((sc, vs))
    return reqs


def _batch(reqs):
    clouds = [B.cloud_from_arrays(sc) for sc, _ in reqs]
    groups = [B.ViewGroup.of([B.views_from_arrays(v) for v in vs]) for _, vs in reqs]
    return B.Batch(clouds, groups)


def test_batched_requests_match_single_renders():
    reqs = _requests()
    cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
    ws, wsb = B.Workspace(), B.Workspace()
    batch = _batch(reqs)
    img, tf, nl = B.render_batched(batch, cfg, wsb)
    w = torch.linspace(-1, 1, batch.pixels, device="cuda")
    g = B.render_batched_backward(batch, cfg, wsb, w, tf, nl)
    torch.cuda.synchronize()
    g_off = np.concatenate([[0], np.cumsum(batch.n)])
    iso_off = np.concatenate([[0], np.cumsum(batch.n_iso)])
    dir_off = np.concatenate([[0], np.cumsum(batch.n - batch.n_iso)])
    v0 = 0
    for r, (sc, vs) in enumerate(reqs):
        cloud = B.cloud_from_arrays(sc)
        acc = None
        poses = []
        for j, v in enumerate(vs):
            gv = B.views_from_arrays(v)
            im, t1, n1 = B.render(cloud, gv, cfg, ws)
            torch.cuda.synchronize()
            assert torch.equal(batch.view_slice(img, v0 + j), im[0])
            assert torch.equal(batch.view_slice(tf, v0 + j), t1[0])
            assert torch.equal(batch.view_slice(nl, v0 + j), n1[0])
            wv = batch.view_slice(w, v0 + j).reshape(1, v.height, v.width).contiguous()
            gs = {k: t.clone() for k, t in B.render_backward(cloud, gv, cfg, ws, wv, t1, n1).items()}
            poses.append(gs.pop("world_to_cam"))
            acc = gs if acc is None else {k: acc[k] + gs[k] for k in acc}
        torch.cuda.synchronize()
        if vs and sc.n:
            a, b_ = g_off[r], g_off[r + 1]
            got = {"means": g["means"][a:b_], "log_scales": g["log_scales"][a:b_],
                   "quats": g["quats"][a:b_], "opacity_logits": g["opacity_logits"][a:b_],
                   "feat_iso": g["feat_iso"][iso_off[r]:iso_off[r + 1]],
                   "feat_dir": g["feat_dir"][dir_off[r]:dir_off[r + 1]],
                   "b_iso": g["b_iso"][r], "B_dir": g["B_dir"][r],
                   "pose": g["world_to_cam"][v0:v0 + len(vs)]}
            ref = dict(acc)
            ref["pose"] = torch.cat(poses)
            compare_grads({k: t.cpu().numpy() for k, t in got.items()},
                          {k: ref[k].cpu().numpy() for k in got}, list(got), tol=1e-5,
                          zero_ok=list(got))
        elif sc.n:
            a, b_ = g_off[r], g_off[r + 1]
            assert float(g["means"][a:b_].abs().max()) == 0.0
            assert float(g["b_iso"][r].abs().max()) == 0.0
        v0 += len(vs)
    ws.close()
    wsb.close()


def test_batched_matches_oracle_per_request():
    reqs = _requests()
    st = syn.Settings(near_plane=0.2)
    cfg = B.config_from_settings(st)
    batch = _batch(reqs)
    ws = B.Workspace()
    img, tf, nl = B.render_batched(batch, cfg, ws)
    torch.cuda.synchronize()
    v = 0
    for sc, vs in reqs:
        for view in vs:
            check_image(sc, view, st, batch.view_slice(img, v).cpu().numpy()[None],
                        batch.view_slice(tf, v).cpu().numpy()[None])
            v += 1
    ws.close()


def test_empty_batch_and_batch_without_views():
    cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
    ws = B.Workspace()
    sc = syn.uniform_cloud(100, seed=1)
    batch = B.Batch([B.cloud_from_arrays(sc)], [B.ViewGroup.of([])])
    img, tf, nl = B.render_batched(batch, cfg, ws)
    g = B.render_batched_backward(batch, cfg, ws, img, tf, nl)
    torch.cuda.synchronize()
    assert img.numel() == 0 and float(g["means"].abs().max()) == 0.0
    ws.close()


def test_batch_depth_and_tile_variants_agree():
    """The staging depth (and warp-streamed staging) changes only how many list
    entries are loaded per round, never the per-pixel order: images are
    bit-identical."""
    sc = syn.uniform_cloud(3000, seed=41)
    views = syn.Views(np.ascontiguousarray(np.stack([
        syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, 2.0])),
        syn.pose_matrix(syn.rot_x(0.3), np.array([0.0, 0.0, 2.1]))]).astype(np.float32)),
        syn.detector(2, 4.0, 8.0 / 90), 77, 90)
    cloud, gv = B.cloud_from_arrays(sc), B.views_from_arrays(views)
    ws = B.Workspace()
    images = []
    for tile in (8, 16, 32):
        st = syn.Settings(near_plane=0.2, tile=tile)
        outs = []
        for depth in (32, 128, 256, 512):  # 32: warp-streamed
            img, tf, nl = B.render(cloud, gv, B.config_from_settings(st, batch_depth=depth), ws)
            outs.append((img.clone(), tf.clone(), nl.clone()))
        torch.cuda.synchronize()
        for o in outs[1:]:
            for a, b in zip(outs[0], o):
                assert torch.equal(a, b), tile
        images.append(outs[0][:2])
    # the tiling changes which lists hold a Gaussian, not which Gaussians
    # contribute to a pixel nor their order: image and T agree across tiles
    for other in images[1:]:
        assert torch.equal(other[0], images[0][0]) and torch.equal(other[1], images[0][1])
    ws.close()


def test_request_times_are_reported():
    reqs = _requests()
    cfg = B.config_from_settings(syn.Settings(near_plane=0.2))
    batch = _batch(reqs)
    ws = B.Workspace()
    img, tf, nl = B.render_batched(batch, cfg, ws)
    B.render_batched_backward(batch, cfg, ws, torch.ones_like(img), tf, nl, want=["world_to_cam"])
    f, b = ws.request_times(batch.n_requests)
    for r, (sc, vs) in enumerate(reqs):
        if vs:
            assert 0 < f[r] < b[r] < 10**10, (r, f[r], b[r])
        else:
            assert f[r] == 0 and b[r] == 0
    ws.close()
