"""Thin Python binding of libddgs.so (include/ddgs.h): argument marshalling only.

Every step of rendering and differentiation runs in the library's CUDA
kernels; this module passes raw device pointers, sizes and the current torch
CUDA stream across the C ABI. There is no CPU fallback: if the library is not
built, or no sm_103 GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np
import torch

from . import build as _build

_lib = None

DDGS_OK = 0
_STATUS = {0: "ok", 1: "invalid argument", 2: "pair capacity exceeded", 3: "non-finite value",
           4: "device wait timed out", 5: "CUDA error", 6: "unsupported device",
           7: "out of device memory"}

# Every symbol include/ddgs.h declares.
EXPORTS = ["ddgs_workspace_create", "ddgs_workspace_destroy", "ddgs_workspace_reserve",
           "ddgs_render", "ddgs_render_backward", "ddgs_l1_loss", "ddgs_workspace_pairs",
           "ddgs_debug_binning", "ddgs_sync_status", "ddgs_parameter_count",
           "ddgs_status_string", "ddgs_last_cuda_error", "ddgs_device_supported",
           "ddgs_kernel_launches", "ddgs_profiler_enable", "ddgs_profiler_collect",
           "ddgs_profiler_kernel_name", "ddgs_render_static", "ddgs_render_batched",
           "ddgs_render_batched_backward", "ddgs_request_times", "ddgs_rads"]


class DDGSError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = f"{what}: {_STATUS.get(code, code)}"
        if code == 5 and _lib is not None:
            msg += f" ({_lib.ddgs_last_cuda_error().decode()})"
        super().__init__(msg)
        self.code = code


class _Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_iso", C.c_int64), ("means", C.c_void_p),
                ("log_scales", C.c_void_p), ("quats", C.c_void_p), ("opacity_logits", C.c_void_p),
                ("feat_iso", C.c_void_p), ("feat_dir", C.c_void_p), ("feat_dir_bf16", C.c_int32),
                ("b_iso", C.c_void_p), ("B_dir", C.c_void_p), ("feat_dim", C.c_int32),
                ("sh_degree", C.c_int32), ("entangled", C.c_int32), ("per_pixel", C.c_int32)]


class _Views(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("world_to_cam", C.c_void_p), ("detector", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("dilation", C.c_float), ("near_plane", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float),
                ("q_max", C.c_float), ("no_sync", C.c_int32), ("batch_depth", C.c_int32)]


class _Batch(C.Structure):
    _fields_ = [("n_requests", C.c_int32), ("gaussian_counts", C.c_void_p),
                ("iso_counts", C.c_void_p), ("view_counts", C.c_void_p), ("heights", C.c_void_p),
                ("widths", C.c_void_p), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("feat_iso", C.c_void_p),
                ("feat_dir", C.c_void_p), ("feat_dir_bf16", C.c_int32), ("b_iso", C.c_void_p),
                ("B_dir", C.c_void_p), ("world_to_cam", C.c_void_p), ("detector", C.c_void_p),
                ("feat_dim", C.c_int32), ("sh_degree", C.c_int32), ("entangled", C.c_int32),
                ("per_pixel", C.c_int32)]


class _Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("feat_iso", C.c_void_p), ("feat_dir", C.c_void_p),
                ("b_iso", C.c_void_p), ("B_dir", C.c_void_p), ("world_to_cam", C.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libddgs.so (it must have been built; see build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libddgs.so is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.ddgs_workspace_create.argtypes = [C.POINTER(vp)]
    lib.ddgs_workspace_destroy.argtypes = [vp]
    lib.ddgs_workspace_reserve.argtypes = [vp, i64, i64, i64]
    lib.ddgs_render.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ddgs_render_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ddgs_l1_loss.argtypes = [vp, vp, i32, i32, i64, vp, vp, vp]
    lib.ddgs_workspace_pairs.argtypes = [vp, C.POINTER(i64)]
    lib.ddgs_debug_binning.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ddgs_sync_status.argtypes = [vp, vp]
    lib.ddgs_parameter_count.argtypes = [i64, i32, i32]
    lib.ddgs_parameter_count.restype = i64
    lib.ddgs_status_string.argtypes = [i32]
    lib.ddgs_status_string.restype = C.c_char_p
    lib.ddgs_last_cuda_error.restype = C.c_char_p
    lib.ddgs_device_supported.restype = i32
    lib.ddgs_render_batched.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.ddgs_render_batched_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ddgs_request_times.argtypes = [vp, vp, vp, vp]
    lib.ddgs_rads.argtypes = [vp, i32, i32, C.c_uint64, vp, vp, vp, vp, vp, vp, vp]
    lib.ddgs_kernel_launches.restype = i64
    lib.ddgs_profiler_enable.argtypes = [i32]
    lib.ddgs_profiler_collect.argtypes = [i32, vp, vp, vp]
    lib.ddgs_profiler_kernel_name.argtypes = [i32]
    lib.ddgs_profiler_kernel_name.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("ddgs_parameter_count", "ddgs_status_string", "ddgs_last_cuda_error",
                        "ddgs_device_supported", "ddgs_kernel_launches",
                        "ddgs_profiler_kernel_name"):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(code: int, what: str):
    if code != DDGS_OK:
        raise DDGSError(code, what)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"tensor on {t.device}, but the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _expect(t: torch.Tensor, name: str, shape, dtypes=(torch.float32,)):
    """The library reads raw pointers with sizes taken from the counts, so a
    tensor of another shape or dtype would be read out of bounds: refuse it."""
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype}, expected one of {tuple(dtypes)}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")


@dataclasses.dataclass
class Cloud:
    """Device tensors of a Gaussian cloud (layouts of ddgs_gaussians)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    feat_iso: torch.Tensor
    feat_dir: torch.Tensor
    b_iso: torch.Tensor
    B_dir: torch.Tensor
    # Eq. 3 variants: both terms in every Gaussian (direct-entangled, Table 3);
    # harmonics evaluated at each pixel's ray direction
    entangled: bool = False
    per_pixel: bool = False

    @property
    def n(self):
        return self.means.shape[0]

    @property
    def n_iso(self):
        return self.feat_iso.shape[0]

    @property
    def feat_dim(self):
        return int(self.b_iso.shape[-1])

    @property
    def sh_degree(self):
        return {3: 1, 8: 2, 15: 3}[int(self.B_dir.shape[-2])]

    def validate(self):
        n, ni, k = self.n, self.n_iso, self.feat_dim
        _expect(self.means, "means", (n, 3))
        _expect(self.log_scales, "log_scales", (n, 3))
        _expect(self.quats, "quats", (n, 4))
        _expect(self.opacity_logits, "opacity_logits", (n,))
        _expect(self.feat_iso, "feat_iso", (ni, k))
        _expect(self.feat_dir, "feat_dir", (n - ni, k), (torch.float32, torch.bfloat16))
        _expect(self.b_iso, "b_iso", (k,))
        if self.B_dir.dim() != 2 or int(self.B_dir.shape[0]) not in (3, 8, 15):
            raise ValueError(f"B_dir: shape {tuple(self.B_dir.shape)}, expected (L(L+2), {k})")
        _expect(self.B_dir, "B_dir", (self.B_dir.shape[0], k))

    def struct(self) -> _Gaussians:
        self.validate()
        bf16 = self.feat_dir.dtype == torch.bfloat16
        return _Gaussians(self.n, self.n_iso, _ptr(self.means), _ptr(self.log_scales),
                          _ptr(self.quats), _ptr(self.opacity_logits),
                          _ptr(self.feat_iso) if self.n_iso else None,
                          _ptr(self.feat_dir) if self.n > self.n_iso else None, int(bf16),
                          _ptr(self.b_iso), _ptr(self.B_dir), self.feat_dim, self.sh_degree,
                          int(self.entangled), int(self.per_pixel))


@dataclasses.dataclass
class Views:
    world_to_cam: torch.Tensor  # [V,3,4] float32, device
    detector: torch.Tensor      # [V,5] float32, device
    height: int
    width: int

    @property
    def n_views(self):
        return self.world_to_cam.shape[0]

    def validate(self):
        V = self.n_views
        _expect(self.world_to_cam, "world_to_cam", (V, 3, 4))
        _expect(self.detector, "detector", (V, 5))

    def struct(self) -> _Views:
        self.validate()
        return _Views(self.n_views, self.height, self.width, _ptr(self.world_to_cam),
                      _ptr(self.detector))


@dataclasses.dataclass
class Config:
    near_plane: float
    tile: int = 16
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    q_max: float = 9.0
    no_sync: bool = False
    batch_depth: int = 256

    def struct(self) -> _Config:
        return _Config(self.tile, self.dilation, self.near_plane, self.alpha_min,
                       self.alpha_max, self.t_min, self.q_max, int(self.no_sync),
                       int(self.batch_depth))


def cloud_from_arrays(scene, device="cuda", feat_dir_bf16: Optional[bool] = None) -> Cloud:
    """Copy a synthetic Scene (numpy float32 arrays) to device tensors."""
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    bf = scene.feat_dir_bf16 if feat_dir_bf16 is None else feat_dir_bf16
    fd = t(scene.feat[scene.n_iso:])
    if bf:
        fd = fd.to(torch.bfloat16)
    return Cloud(t(scene.means), t(scene.log_scales), t(scene.quats), t(scene.opacity_logits),
                 t(scene.feat[:scene.n_iso]), fd.contiguous(), t(scene.b_iso), t(scene.B_dir),
                 bool(scene.entangled), bool(scene.per_pixel))


def views_from_arrays(views, device="cuda") -> Views:
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    return Views(t(views.world_to_cam), t(views.detector), views.height, views.width)


def config_from_settings(st, no_sync=False, batch_depth=256) -> Config:
    return Config(near_plane=st.near_plane, tile=st.tile, dilation=st.dilation,
                  alpha_min=st.alpha_min, alpha_max=st.alpha_max, t_min=st.t_min,
                  q_max=st.q_max, no_sync=no_sync, batch_depth=batch_depth)


class Workspace:
    """Library-owned device workspace (sort buffers, records, status word)."""

    def __init__(self):
        lib = load()
        h = C.c_void_p()
        _check(lib.ddgs_workspace_create(C.byref(h)), "ddgs_workspace_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def reserve(self, records: int, pairs: int, tiles: int):
        _check(load().ddgs_workspace_reserve(self._h, records, pairs, tiles),
               "ddgs_workspace_reserve")

    def pairs(self) -> int:
        m = C.c_int64()
        _check(load().ddgs_workspace_pairs(self._h, C.byref(m)), "ddgs_workspace_pairs")
        return m.value

    def request_times(self, n_requests: int):
        """(fwd_ns, bwd_ns) per request of the last batched render + backward."""
        f = np.zeros(n_requests, np.uint64)
        b = np.zeros(n_requests, np.uint64)
        _check(load().ddgs_request_times(self._h, f.ctypes.data, b.ctypes.data, _stream()),
               "ddgs_request_times")
        return f, b

    def sync_status(self) -> int:
        return load().ddgs_sync_status(self._h, _stream())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ddgs_workspace_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render(cloud: Cloud, views: Views, cfg: Config, ws: Workspace, out=None):
    """ddgs_render: returns (image, t_final, n_last), each [V, H, W]."""
    lib = load()
    V, H, W = views.n_views, views.height, views.width
    dev = cloud.means.device
    if out is None:
        out = (torch.empty((V, H, W), dtype=torch.float32, device=dev),
               torch.empty((V, H, W), dtype=torch.float32, device=dev),
               torch.empty((V, H, W), dtype=torch.int32, device=dev))
    img, tf, nl = out
    _expect(img, "image", (V, H, W))
    _expect(tf, "t_final", (V, H, W))
    _expect(nl, "n_last", (V, H, W), (torch.int32,))
    g, v, c = cloud.struct(), views.struct(), cfg.struct()
    _check(lib.ddgs_render(C.byref(g), C.byref(v), C.byref(c), ws.handle, _ptr(img), _ptr(tf),
                           _ptr(nl), _stream()), "ddgs_render")
    return img, tf, nl


GRAD_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "feat_iso", "feat_dir", "b_iso",
               "B_dir", "world_to_cam")


def render_backward(cloud: Cloud, views: Views, cfg: Config, ws: Workspace, dL_dimage, t_final,
                    n_last, want=GRAD_FIELDS, out=None):
    """ddgs_render_backward: returns a dict of float32 gradients for `want`."""
    lib = load()
    dev = cloud.means.device
    shapes = dict(means=cloud.means.shape, log_scales=cloud.log_scales.shape,
                  quats=cloud.quats.shape, opacity_logits=cloud.opacity_logits.shape,
                  feat_iso=cloud.feat_iso.shape, feat_dir=cloud.feat_dir.shape,
                  b_iso=cloud.b_iso.shape, B_dir=cloud.B_dir.shape,
                  world_to_cam=views.world_to_cam.shape)
    grads = dict(out or {})
    for k in want:
        if k not in grads:
            grads[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
    for k, t in grads.items():
        _expect(t, f"gradient {k}", shapes[k])
    img_shape = (views.n_views, views.height, views.width)
    _expect(dL_dimage, "dL_dimage", img_shape)
    _expect(t_final, "t_final", img_shape)
    _expect(n_last, "n_last", img_shape, (torch.int32,))
    gs = _Grads(*[_ptr(grads[k]) if k in grads else None for k in GRAD_FIELDS])
    g, v, c = cloud.struct(), views.struct(), cfg.struct()
    _check(lib.ddgs_render_backward(C.byref(g), C.byref(v), C.byref(c), ws.handle,
                                    _ptr(dL_dimage.contiguous()), _ptr(t_final), _ptr(n_last),
                                    C.byref(gs), _stream()), "ddgs_render_backward")
    return grads


def l1_loss(image: torch.Tensor, target: torch.Tensor, loss=None, grad=None):
    """ddgs_l1_loss: per-view mean |image - target| and its gradient."""
    lib = load()
    V = image.shape[0]
    hw = image[0].numel()
    per_view = int(target.dim() == image.dim() and target.shape[0] == V and V > 1)
    loss = torch.empty(V, dtype=torch.float32, device=image.device) if loss is None else loss
    grad = torch.empty_like(image) if grad is None else grad
    _expect(image, "image", image.shape)
    if target.dtype != torch.float32 or target.numel() != (V * hw if per_view else hw):
        raise ValueError(f"target: {tuple(target.shape)} {target.dtype}, expected float32 with "
                         f"{V * hw if per_view else hw} elements")
    _expect(loss, "loss", (V,))
    _expect(grad, "grad", image.shape)
    _check(lib.ddgs_l1_loss(_ptr(image), _ptr(target.contiguous()), per_view, V, hw, _ptr(loss),
                            _ptr(grad), _stream()), "ddgs_l1_loss")
    return loss, grad


def debug_binning(ws: Workspace, n_views: int, n: int, n_tiles: int):
    """Copies of the last render's binning: tiles_touched [V,n], keys, vals, ranges [tiles,2]."""
    lib = load()
    torch.cuda.current_stream().synchronize()
    m = ws.pairs()
    dev = "cuda"
    tt = torch.empty((n_views, n), dtype=torch.int32, device=dev)
    keys = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
    vals = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    rng = torch.empty((n_tiles, 2), dtype=torch.int32, device=dev)
    _check(lib.ddgs_debug_binning(ws.handle, _ptr(tt), _ptr(keys), _ptr(vals), _ptr(rng),
                                  _stream()), "ddgs_debug_binning")
    torch.cuda.current_stream().synchronize()
    return dict(tiles_touched=tt.cpu().numpy().view(np.uint32), keys=keys[:m].cpu().numpy().view(np.uint64),
                vals=vals[:m].cpu().numpy().view(np.uint32), ranges=rng.cpu().numpy().view(np.uint32), m=m)


def kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return int(load().ddgs_kernel_launches())


def profiler_enable(on: bool = True):
    _check(load().ddgs_profiler_enable(int(on)), "ddgs_profiler_enable")


def profiler_collect() -> dict:
    """{kernel name: (total ms, launches)} since the last collect; resets."""
    lib = load()
    n = 64
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    nk = C.c_int32()
    _check(lib.ddgs_profiler_collect(n, C.addressof(ms), C.addressof(cnt), C.addressof(nk)),
           "ddgs_profiler_collect")
    return {lib.ddgs_profiler_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(nk.value)
            if cnt[i] > 0}


def parameter_count(n: int, k: int = 8, L: int = 1) -> int:
    return int(load().ddgs_parameter_count(n, k, L))


def device_supported() -> bool:
    return bool(load().ddgs_device_supported())


class RenderFunction(torch.autograd.Function):
    """torch.autograd.Function over ddgs_render / ddgs_render_backward.

    Inputs: the cloud's tensors and the poses; returns the image [V, H, W].
    The backward recomputes the blending state from the workspace's sorted
    lists (it must run before the next render on the same workspace).
    `variant` = (entangled, per_pixel) selects an Eq. 3 variant."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, feat_iso, feat_dir, b_iso, B_dir,
                world_to_cam, detector, height, width, cfg, ws, variant=(False, False)):
        cloud = Cloud(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                      opacity_logits.contiguous(), feat_iso.contiguous(), feat_dir.contiguous(),
                      b_iso.contiguous(), B_dir.contiguous(), bool(variant[0]), bool(variant[1]))
        views = Views(world_to_cam.contiguous(), detector.contiguous(), height, width)
        img, tf, nl = render(cloud, views, cfg, ws)
        ctx.cloud, ctx.views, ctx.cfg, ctx.ws = cloud, views, cfg, ws
        ctx.save_for_backward(tf, nl)
        ctx.feat_dir_dtype = feat_dir.dtype
        ctx.mark_non_differentiable(tf, nl)
        return img, tf, nl

    @staticmethod
    def backward(ctx, g_img, g_tf, g_nl):
        tf, nl = ctx.saved_tensors
        names = ["means", "log_scales", "quats", "opacity_logits", "feat_iso", "feat_dir",
                 "b_iso", "B_dir", "world_to_cam"]
        want = [n for n, need in zip(names, ctx.needs_input_grad[:9]) if need]
        g = render_backward(ctx.cloud, ctx.views, ctx.cfg, ctx.ws, g_img.contiguous(), tf, nl,
                            want=want)
        out = [g.get(n) for n in names]
        if out[5] is not None and ctx.feat_dir_dtype != torch.float32:
            out[5] = out[5].to(ctx.feat_dir_dtype)
        return (*out, None, None, None, None, None, None)


def render_differentiable(cloud: Cloud, views: Views, cfg: Config, ws: Workspace):
    """Autograd-aware render; returns (image, t_final, n_last)."""
    return RenderFunction.apply(cloud.means, cloud.log_scales, cloud.quats, cloud.opacity_logits,
                                cloud.feat_iso, cloud.feat_dir, cloud.b_iso, cloud.B_dir,
                                views.world_to_cam, views.detector, views.height, views.width,
                                cfg, ws)


@dataclasses.dataclass
class ViewGroup:
    """The views of one request of a batch; each view has its own detector size."""
    world_to_cam: torch.Tensor  # [Vr,3,4] float32, device
    detector: torch.Tensor      # [Vr,5] float32, device
    sizes: list                 # [(H, W)] per view

    @property
    def n_views(self):
        return len(self.sizes)

    def validate(self):
        V = self.n_views
        _expect(self.world_to_cam, "world_to_cam", (V, 3, 4))
        _expect(self.detector, "detector", (V, 5))

    @staticmethod
    def of(views_list, device="cuda"):
        """From a list of single-size Views (device tensors)."""
        if not views_list:
            return ViewGroup(torch.empty((0, 3, 4), device=device), torch.empty((0, 5), device=device), [])
        return ViewGroup(torch.cat([v.world_to_cam for v in views_list]).contiguous(),
                         torch.cat([v.detector for v in views_list]).contiguous(),
                         [(v.height, v.width) for v in views_list for _ in range(v.n_views)])


def _sizes(v):
    return list(v.sizes) if isinstance(v, ViewGroup) else [(v.height, v.width)] * v.n_views


class Batch:
    """Device tensors of a batch of requests (ddgs_batch): concatenated clouds,
    per-request bases, per-view poses and detectors, host count arrays.
    `views[r]` is a Views (one size) or a ViewGroup (per-view sizes)."""

    def __init__(self, clouds, views):
        if len(clouds) != len(views):
            raise ValueError(f"{len(clouds)} clouds but {len(views)} view sets")
        for c in clouds:
            c.validate()
        for v in views:
            v.validate()
        self.clouds, self.views = clouds, views
        self.means = torch.cat([c.means for c in clouds]).contiguous()
        self.log_scales = torch.cat([c.log_scales for c in clouds]).contiguous()
        self.quats = torch.cat([c.quats for c in clouds]).contiguous()
        self.opacity_logits = torch.cat([c.opacity_logits for c in clouds]).contiguous()
        self.feat_iso = torch.cat([c.feat_iso for c in clouds]).contiguous()
        self.feat_dir = torch.cat([c.feat_dir for c in clouds]).contiguous()
        self.b_iso = torch.stack([c.b_iso for c in clouds]).contiguous()
        self.B_dir = torch.stack([c.B_dir for c in clouds]).contiguous()
        self.world_to_cam = torch.cat([v.world_to_cam for v in views]).contiguous()
        self.detector = torch.cat([v.detector for v in views]).contiguous()
        self.n = np.array([c.n for c in clouds], np.int64)
        self.n_iso = np.array([c.n_iso for c in clouds], np.int64)
        self.nv = np.array([v.n_views for v in views], np.int32)
        sizes = [hw for v in views for hw in _sizes(v)]
        self.H = np.array([h for h, _ in sizes] or [0], np.int32)[:len(sizes)]
        self.W = np.array([w for _, w in sizes] or [0], np.int32)[:len(sizes)]
        self.pixel_offsets = np.concatenate([[0], np.cumsum(self.H.astype(np.int64) * self.W)])

    @property
    def n_requests(self):
        return len(self.clouds)

    @property
    def pixels(self):
        return int(self.pixel_offsets[-1])

    def struct(self) -> _Batch:
        bf16 = self.feat_dir.dtype == torch.bfloat16
        R = self.n_requests
        p = lambda t: _ptr(t) if t.numel() else None
        c0 = self.clouds[0] if self.clouds else None
        return _Batch(R, self.n.ctypes.data, self.n_iso.ctypes.data, self.nv.ctypes.data,
                      self.H.ctypes.data, self.W.ctypes.data, p(self.means), p(self.log_scales),
                      p(self.quats), p(self.opacity_logits), p(self.feat_iso), p(self.feat_dir),
                      int(bf16), p(self.b_iso), p(self.B_dir), p(self.world_to_cam), p(self.detector),
                      c0.feat_dim if c0 else 8, c0.sh_degree if c0 else 1,
                      int(c0.entangled) if c0 else 0, int(c0.per_pixel) if c0 else 0)

    def view_slice(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        a, b = int(self.pixel_offsets[v]), int(self.pixel_offsets[v + 1])
        return flat[a:b].view(int(self.H[v]), int(self.W[v]))


def render_batched(batch: Batch, cfg: Config, ws: Workspace, out=None):
    """ddgs_render_batched: flat (image, t_final, n_last) over all views."""
    lib = load()
    P = batch.pixels
    dev = batch.means.device
    if out is None:
        out = (torch.empty(P, dtype=torch.float32, device=dev),
               torch.empty(P, dtype=torch.float32, device=dev),
               torch.empty(P, dtype=torch.int32, device=dev))
    img, tf, nl = out
    _expect(img, "image", (P,))
    _expect(tf, "t_final", (P,))
    _expect(nl, "n_last", (P,), (torch.int32,))
    b, c = batch.struct(), cfg.struct()
    _check(lib.ddgs_render_batched(C.byref(b), C.byref(c), ws.handle, _ptr(img), _ptr(tf),
                                   _ptr(nl), _stream()), "ddgs_render_batched")
    return img, tf, nl


def render_batched_backward(batch: Batch, cfg: Config, ws: Workspace, dL_dimage, t_final, n_last,
                            want=GRAD_FIELDS, out=None):
    lib = load()
    dev = batch.means.device
    shapes = dict(means=batch.means.shape, log_scales=batch.log_scales.shape,
                  quats=batch.quats.shape, opacity_logits=batch.opacity_logits.shape,
                  feat_iso=batch.feat_iso.shape, feat_dir=batch.feat_dir.shape,
                  b_iso=batch.b_iso.shape, B_dir=batch.B_dir.shape,
                  world_to_cam=batch.world_to_cam.shape)
    grads = dict(out or {})
    for k in want:
        if k not in grads:
            grads[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
    for k, t in grads.items():
        _expect(t, f"gradient {k}", shapes[k])
    P = batch.pixels
    _expect(dL_dimage, "dL_dimage", (P,))
    _expect(t_final, "t_final", (P,))
    _expect(n_last, "n_last", (P,), (torch.int32,))
    gs = _Grads(*[(_ptr(grads[k]) if grads[k].numel() else None) if k in grads else None
                  for k in GRAD_FIELDS])
    b, c = batch.struct(), cfg.struct()
    _check(lib.ddgs_render_batched_backward(C.byref(b), C.byref(c), ws.handle,
                                            _ptr(dL_dimage.contiguous()), _ptr(t_final),
                                            _ptr(n_last), C.byref(gs), _stream()),
           "ddgs_render_batched_backward")
    return grads


class _Volume(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("hu", C.c_void_p),
                ("spacing", C.c_float * 3), ("origin", C.c_float * 3)]


def rads(hu: torch.Tensor, spacing, origin, n1: int = 15000, n2: int = 10000, seed: int = 0,
         ws: Optional[Workspace] = None, debug: bool = False) -> dict:
    """ddgs_rads (Sec. 3.3): the initial cloud of a CT volume hu [nz, ny, nx]
    (int16 HU, device). Returns means [n, 3], log_scales [n, 3], n_iso and the
    counts; with debug, also the kept edge ids and drawn voxel indices."""
    lib = load()
    assert hu.dtype == torch.int16 and hu.dim() == 3 and hu.is_contiguous()
    nz, ny, nx = hu.shape
    dev = hu.device
    vol = _Volume(nx, ny, nz, _ptr(hu), (C.c_float * 3)(*spacing), (C.c_float * 3)(*origin))
    n = max(n1 + n2, 1)
    means = torch.empty((n, 3), dtype=torch.float32, device=dev)
    log_scales = torch.empty((n, 3), dtype=torch.float32, device=dev)
    kept = torch.empty(max(n1, 1), dtype=torch.int64, device=dev) if debug else None
    draws = torch.empty(max(n2, 1), dtype=torch.int64, device=dev) if debug else None
    counts = (C.c_int64 * 3)()
    own = ws is None
    ws = ws or Workspace()
    try:
        _check(lib.ddgs_rads(C.byref(vol), n1, n2, C.c_uint64(seed & (2 ** 64 - 1)), ws.handle,
                             _ptr(means), _ptr(log_scales), _ptr(kept), _ptr(draws),
                             C.addressof(counts), _stream()), "ddgs_rads")
    finally:
        if own:
            torch.cuda.current_stream().synchronize()
            ws.close()
    m1, m2, M = int(counts[0]), int(counts[1]), int(counts[2])
    out = dict(means=means[:m1 + m2], log_scales=log_scales[:m1 + m2], n_mc=m1, n_dw=m2,
               n_crossings=M, n_iso=m1 + m2 - m2 // 2)
    if debug:
        out["kept_edges"] = kept[:m1]
        out["draw_voxels"] = draws[:m2]
    return out

