"""2D/3D pose registration by gradient descent through the renderer (Sec. 4.3).

A pose is estimated by rendering the cloud at the current pose, comparing the
rendering with the target X-ray (L1, the l1 term of Eq. 2), back-propagating
to the pose and stepping Adam (learning rate 0.05), starting from the
isocenter pose. Many candidates are registered at once: each is one view of a
single batched render, so every iteration is one ddgs_render, one
ddgs_l1_loss and one ddgs_render_backward for all candidates. After a few
eager iterations the whole iteration (pose map, render, loss, backward, Adam
step) is captured once in a CUDA graph and replayed; the renders then run in
no-sync mode on a workspace reserved for 1.5x the initial pair count.

The pose is a 6-DoF correction (rotation vector w in units of `rot_unit`
radians, translation d in units of `trans_unit` millimetres) applied about the
isocenter on top of the initial pose: world_to_cam = [R0 exp([w]x) | R0 d + t0].
The paper gives the learning rate (0.05) but not the units of its pose
parameters; with 0.1 rad and 10 mm units one Adam step moves a pose by about
0.3 degrees and 0.5 mm. The small map from (w, d) to
the 3x4 matrix is differentiated by torch; everything per pixel and per
Gaussian runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import binding as B


def _skew(w: torch.Tensor) -> torch.Tensor:
    z = torch.zeros_like(w[..., 0])
    return torch.stack([torch.stack([z, -w[..., 2], w[..., 1]], -1),
                        torch.stack([w[..., 2], z, -w[..., 0]], -1),
                        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def rodrigues(w: torch.Tensor) -> torch.Tensor:
    """Rotation matrices exp([w]x) for rotation vectors w [..., 3] (float64 math)."""
    th2 = (w * w).sum(-1, keepdim=True).unsqueeze(-1)
    big = th2 > 1e-12
    # both branches of a where() are differentiated: keep the unused one finite
    th2s = torch.where(big, th2, torch.ones_like(th2))
    th = torch.sqrt(th2s)
    K = _skew(w)
    a = torch.where(big, torch.sin(th) / th, 1 - th2 / 6)
    b = torch.where(big, (1 - torch.cos(th)) / th2s, 0.5 - th2 / 24)
    eye = torch.eye(3, dtype=w.dtype, device=w.device).expand(K.shape)
    return eye + a * K + b * (K @ K)


def compose(R0: torch.Tensor, t0: torch.Tensor, w: torch.Tensor, d: torch.Tensor,
            trans_unit: float, rot_unit: float = 1.0) -> torch.Tensor:
    """world_to_cam [V,3,4] for corrections (w, d) about the isocenter."""
    R = R0 @ rodrigues(w * rot_unit)
    t = t0 + (R0 @ (d * trans_unit).unsqueeze(-1)).squeeze(-1)
    return torch.cat([R, t.unsqueeze(-1)], -1)


def rotation_error_deg(Ra: np.ndarray, Rb: np.ndarray) -> np.ndarray:
    """Angular distance between rotations [..., 3, 3], degrees."""
    M = np.einsum("...ji,...jk->...ik", Ra, Rb)
    c = np.clip((np.trace(M, axis1=-2, axis2=-1) - 1) / 2, -1.0, 1.0)
    return np.degrees(np.arccos(c))


def translation_error_mm(Ta: np.ndarray, Tb: np.ndarray) -> np.ndarray:
    """Distance between the isocenter's camera-frame positions (t) of two poses, mm."""
    return np.linalg.norm(Ta[..., 3] - Tb[..., 3], axis=-1)


class _L1(torch.autograd.Function):
    """Per-view mean |image - target| through ddgs_l1_loss (a library kernel)."""

    @staticmethod
    def forward(ctx, image, target):
        loss, grad = B.l1_loss(image.contiguous(), target)
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        (grad,) = ctx.saved_tensors
        return grad * g_loss.view(-1, 1, 1), None


@dataclasses.dataclass
class RegistrationResult:
    poses: np.ndarray          # [V,3,4] final estimates
    rot_err_deg: np.ndarray    # [V] against the true poses (if given)
    trans_err_mm: np.ndarray   # [V]
    loss: np.ndarray           # [iters, V]


_EAGER_ITERS = 3  # iterations run before the capture (also the capture's warm-up)


class _Adam:
    """Adam (Kingma & Ba) on a list of tensors with device-side state, so that a
    step can be captured in a CUDA graph: m <- b1 m + (1 - b1) g,
    v <- b2 v + (1 - b2) g^2, p <- p - lr m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, params, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.params, self.lr, self.b1, self.b2, self.eps = list(params), lr, b1, b2, eps
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.t = torch.zeros((), dtype=torch.float64, device=self.params[0].device)

    def zero_grad(self):
        for p in self.params:
            if p.grad is not None:
                p.grad.zero_()

    @torch.no_grad()
    def step(self):
        self.t += 1
        c1 = 1 - torch.pow(self.b1, self.t)
        c2 = 1 - torch.pow(self.b2, self.t)
        for p, m, v in zip(self.params, self.m, self.v):
            g = p.grad
            m.mul_(self.b1).add_(g, alpha=1 - self.b1)
            v.mul_(self.b2).addcmul_(g, g, value=1 - self.b2)
            p.sub_(self.lr * (m / c1) / (torch.sqrt(v / c2) + self.eps))


def coarse_targets(targets: torch.Tensor, scale: int, blur_px2: float) -> torch.Tensor:
    """Targets [V,H,W] for a coarse stage: means over scale x scale pixel
    blocks, then a Gaussian blur of variance blur_px2 (coarse pixels^2) with
    replicated edges. A preprocessing of the fixed target images, once per
    stage; the renders of every iteration run in the library's kernels."""
    t = targets.unsqueeze(1)
    if scale > 1:
        t = torch.nn.functional.avg_pool2d(t, scale)
    if blur_px2 > 0:
        r = int(math.ceil(3 * math.sqrt(blur_px2)))
        x = torch.arange(-r, r + 1, dtype=t.dtype, device=t.device)
        k = torch.exp(-0.5 * x * x / blur_px2)
        k = k / k.sum()
        pad = torch.nn.functional.pad
        t = torch.nn.functional.conv2d(pad(t, (r, r, 0, 0), mode="replicate"), k.view(1, 1, 1, -1))
        t = torch.nn.functional.conv2d(pad(t, (0, 0, r, r), mode="replicate"), k.view(1, 1, -1, 1))
    return t.squeeze(1).contiguous()


def register(cloud: B.Cloud, detector: torch.Tensor, height: int, width: int,
             targets: torch.Tensor, init_pose: torch.Tensor, cfg: B.Config,
             iters: int = 200, lr: float = 0.05, trans_unit: float = 10.0,
             rot_unit: float = 0.1, true_poses: np.ndarray | None = None, ws: B.Workspace | None = None,
             graph: bool = True, schedule=None) -> RegistrationResult:
    """Register V candidates at once. targets [V,H,W]; init_pose [V,3,4] or
    [3,4]; detector [V,5]. Adam on (w, d) with learning rate `lr`. With
    graph=True the iterations of a stage after its first few replay one CUDA
    graph; if the pair count ever outgrows the reserved workspace, the stage
    is run again without the graph.

    schedule: stages (iterations, scale, dilation px^2) run in order with one
    Adam state, coarse to fine. A stage renders a detector of
    (height / scale) x (width / scale) pixels of scale times the pitch, with
    the given dilation, against coarse_targets(targets, scale, blur) where the
    blur makes up the difference between that dilation and the full-size
    render's (cfg.dilation / scale^2) and the block mean (1/12 px^2 per axis).
    The default is one stage: (iters, 1, cfg.dilation)."""
    dev = cloud.means.device
    V = targets.shape[0]
    P0 = init_pose.to(dev, torch.float64).expand(V, 3, 4) if init_pose.dim() == 2 else \
        init_pose.to(dev, torch.float64)
    R0, t0 = P0[:, :, :3], P0[:, :, 3]
    w = torch.zeros((V, 3), dtype=torch.float64, device=dev, requires_grad=True)
    d = torch.zeros((V, 3), dtype=torch.float64, device=dev, requires_grad=True)
    opt = _Adam([w, d], lr=lr)
    ws = ws or B.Workspace()
    det = detector.to(dev, torch.float32).expand(V, 5).contiguous()
    schedule = list(schedule) if schedule else [(iters, 1, cfg.dilation)]
    total = sum(int(n) for n, _, _ in schedule)
    losses = torch.zeros((total, V), dtype=torch.float32, device=dev)
    done = 0
    for n_it, scale, dil in schedule:
        n_it, scale = int(n_it), int(scale)
        if n_it <= 0:
            continue
        if height % scale or width % scale:
            raise ValueError("a stage's scale must divide the detector size")
        H_s, W_s = height // scale, width // scale
        det_s = det.clone()
        det_s[:, 1:3] *= scale   # pitch
        det_s[:, 3:5] /= scale   # principal point offsets, pixels
        cfg_s = dataclasses.replace(cfg, dilation=float(dil))
        blur = max(0.0, float(dil) - cfg.dilation / scale ** 2 - (1.0 / 12.0 if scale > 1 else 0.0))
        tgt = coarse_targets(targets, scale, blur) if (scale > 1 or blur > 0) else targets
        _run_stage(cloud, det_s, H_s, W_s, tgt, R0, t0, w, d, opt, cfg_s, n_it, trans_unit,
                   rot_unit, ws, graph, losses[done:done + n_it])
        done += n_it
    with torch.no_grad():
        final = compose(R0, t0, w, d, trans_unit, rot_unit).cpu().numpy()
    if true_poses is not None:
        rot = rotation_error_deg(final[:, :, :3], true_poses[:, :, :3])
        tr = translation_error_mm(final, true_poses)
    else:
        rot = tr = np.full(V, np.nan)
    return RegistrationResult(final, rot, tr, losses.cpu().numpy())


def _run_stage(cloud, det, height, width, targets, R0, t0, w, d, opt, cfg, iters, trans_unit,
               rot_unit, ws, graph, losses):
    """iters Adam iterations of one stage; per-iteration losses into losses."""
    graph = graph and iters > _EAGER_ITERS
    run_cfg = cfg
    state = ([p.detach().clone() for p in (w, d)], [m.clone() for m in opt.m],
             [v.clone() for v in opt.v], opt.t.clone())

    def iteration():
        opt.zero_grad()
        pose = compose(R0, t0, w, d, trans_unit, rot_unit).to(torch.float32).contiguous()
        img, _, _ = B.RenderFunction.apply(cloud.means, cloud.log_scales, cloud.quats,
                                           cloud.opacity_logits, cloud.feat_iso, cloud.feat_dir,
                                           cloud.b_iso, cloud.B_dir, pose, det, height, width,
                                           run_cfg, ws)
        loss = _L1.apply(img, targets)
        loss.sum().backward()
        opt.step()
        return loss.detach()

    if not graph:
        for i in range(iters):
            losses[i].copy_(iteration())
        return
    V = targets.shape[0]
    # size the workspace for no-sync renders from the stage's starting pair count
    with torch.no_grad():
        pose = compose(R0, t0, w, d, trans_unit, rot_unit).to(torch.float32).contiguous()
        B.render(cloud, B.Views(pose, det, height, width), cfg, ws)
    torch.cuda.synchronize()
    tiles = V * (-(-height // cfg.tile)) * (-(-width // cfg.tile))
    ws.reserve(V * cloud.n, int(ws.pairs() * 1.5) + 4096, tiles)
    run_cfg = dataclasses.replace(cfg, no_sync=True)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for i in range(_EAGER_ITERS):
            losses[i].copy_(iteration())
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        loss_static = iteration()
    for i in range(_EAGER_ITERS, iters):
        g.replay()
        losses[i].copy_(loss_static)
    torch.cuda.synchronize()
    del g
    if ws.sync_status() != 0:  # a no-sync render ran out of room: redo the stage without the graph
        with torch.no_grad():
            for p, q in zip((w, d), state[0]):
                p.copy_(q)
            for m, q in zip(opt.m, state[1]):
                m.copy_(q)
            for v, q in zip(opt.v, state[2]):
                v.copy_(q)
            opt.t.copy_(state[3])
        _run_stage(cloud, det, height, width, targets, R0, t0, w, d, opt, cfg, iters, trans_unit,
                   rot_unit, ws, False, losses)


def perturbed_poses(rng: np.random.Generator, base: np.ndarray, n: int, max_deg: float,
                    max_mm: float) -> np.ndarray:
    """n poses: base composed with rotations about the isocenter (rotation
    vector of norm up to max_deg) and translations up to max_mm per axis."""
    out = np.zeros((n, 3, 4))
    for k in range(n):
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        ang = math.radians(rng.uniform(0.5, 1.0) * max_deg)
        wv = torch.tensor(axis * ang, dtype=torch.float64)
        Rk = rodrigues(wv).numpy()
        dk = rng.uniform(-max_mm, max_mm, 3)
        out[k, :, :3] = base[:, :3] @ Rk
        out[k, :, 3] = base[:, 3] + base[:, :3] @ dk
    return out.astype(np.float32)
