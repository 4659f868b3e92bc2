"""Python access to the plain CPU oracle (C, FP64 renderer + FP32 binning reference).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users. The product library never
imports, links or executes anything here, and nothing here calls the library.

Inputs are the float32 arrays of ``paper_2406_02518_gb300.synthetic`` (the
bits the GPU sees); the FP64 renderer widens them exactly to float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "render_f64.c"), os.path.join(_HERE, "binning_f32.c")]
_HDR = os.path.join(_HERE, "ddgs_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, OpenMP, no floating-point contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
        return _OUT
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_iso", C.c_int32), ("k", C.c_int32), ("L", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("feat", C.c_void_p),
                ("b_iso", C.c_void_p), ("B_dir", C.c_void_p),
                ("entangled", C.c_int32), ("per_pixel", C.c_int32)]


class _Views(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("world_to_cam", C.c_void_p), ("detector", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("dilation", C.c_double), ("near_plane", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_min", C.c_double),
                ("q_max", C.c_double)]


class _Geom32(C.Structure):
    _fields_ = [("n", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p)]


class _Views32(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("world_to_cam", C.c_void_p), ("detector", C.c_void_p)]


class _Config32(C.Structure):
    _fields_ = [("tile", C.c_int32), ("dilation", C.c_float), ("near_plane", C.c_float),
                ("q_max", C.c_float)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        vp = C.c_void_p
        _lib.or_render.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
        _lib.or_render_backward.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp, vp] + [vp] * 9 + [C.c_int]
        _lib.or_project.argtypes = [vp, vp, vp, vp]
        _lib.or32_project.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        _lib.or32_bin.argtypes = [vp, vp, C.c_int32, vp, vp, vp, C.c_int64, vp, vp, vp]
        _lib.or_count_inside.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp, C.c_int]
        _lib.or_exp32.argtypes = [C.c_float]
        _lib.or_exp32.restype = C.c_float
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _Pack:
    """Holds the float64 copies (and keeps them alive) for one call."""

    def __init__(self, scene, views, settings):
        self.arrs = dict(means=_d(scene.means), ls=_d(scene.log_scales), q=_d(scene.quats),
                         o=_d(scene.opacity_logits), f=_d(scene.feat), b=_d(scene.b_iso),
                         B=_d(scene.B_dir), T=_d(views.world_to_cam), det=_d(views.detector))
        a = self.arrs
        kl = int(np.asarray(scene.B_dir).shape[0])
        L = {3: 1, 8: 2, 15: 3, 24: 4}[kl]
        self.scene = _Scene(scene.n, scene.n_iso, scene.feat.shape[1], L, _p(a["means"]),
                            _p(a["ls"]), _p(a["q"]), _p(a["o"]), _p(a["f"]), _p(a["b"]),
                            _p(a["B"]), int(bool(scene.entangled)), int(bool(scene.per_pixel)))
        self.views = _Views(views.n_views, views.height, views.width, _p(a["T"]), _p(a["det"]))
        s = settings
        self.cfg = _Config(s.tile, s.dilation, s.near_plane, s.alpha_min, s.alpha_max,
                           s.t_min, s.q_max)


def exp32(x: float) -> float:
    return float(lib().or_exp32(C.c_float(x)))


def project32(scene, views, settings):
    """FP32 binning reference, per (view, Gaussian): depth, tiles touched, rect, aux."""
    V, n = views.n_views, scene.n
    g = _Geom32(n, _p(scene.means), _p(scene.log_scales), _p(scene.quats))
    vw = _Views32(V, views.height, views.width, _p(views.world_to_cam), _p(views.detector))
    cfg = _Config32(settings.tile, settings.dilation, settings.near_plane, settings.q_max)
    for a in (scene.means, scene.log_scales, scene.quats, views.world_to_cam, views.detector):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    depth = np.zeros((V, n), np.float32)
    tt = np.zeros((V, n), np.uint32)
    rect = np.zeros((V, n, 4), np.int32)
    aux = np.zeros((V, n, 4), np.float32)
    rc = lib().or32_project(C.byref(g), C.byref(vw), C.byref(cfg), _p(depth), _p(tt),
                            _p(rect), _p(aux))
    if rc:
        raise RuntimeError(f"or32_project failed ({rc})")
    return dict(depth=depth, tiles_touched=tt, rect=rect, aux=aux)


def bin32(scene, views, settings, proj=None):
    """FP32 binning reference: sorted keys, values, and per-(view, tile) ranges."""
    proj = proj or project32(scene, views, settings)
    V, n = views.n_views, scene.n
    m = int(proj["tiles_touched"].astype(np.int64).sum())
    t = settings.tile
    tiles = ((views.width + t - 1) // t) * ((views.height + t - 1) // t)
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros((V * tiles, 2), np.uint32)
    vw = _Views32(V, views.height, views.width, _p(views.world_to_cam), _p(views.detector))
    cfg = _Config32(t, settings.dilation, settings.near_plane, settings.q_max)
    rc = lib().or32_bin(C.byref(vw), C.byref(cfg), n, _p(proj["depth"]),
                        _p(proj["tiles_touched"]), _p(proj["rect"]), m, _p(keys), _p(vals),
                        _p(ranges))
    if rc:
        raise RuntimeError(f"or32_bin failed ({rc})")
    return dict(keys=keys[:m], vals=vals[:m], ranges=ranges, m=m, **proj)


def project64(scene, views, settings) -> np.ndarray:
    """FP64 projections [V, n, 9] = u, v, conic a, b, c, alpha, color, depth, valid."""
    pk = _Pack(scene, views, settings)
    out = np.zeros((views.n_views, scene.n, 9), np.float64)
    rc = lib().or_project(C.byref(pk.scene), C.byref(pk.views), C.byref(pk.cfg), _p(out))
    if rc:
        raise RuntimeError(f"or_project failed ({rc})")
    return out


def _pix(views, pix):
    if pix is None:
        return None, views.n_views * views.height * views.width
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    return pix, pix.shape[0]


def render(scene, views, settings, pix=None, flip_masks=None, depth32=None, threads=0):
    """FP64 forward of Eq. 1 at every requested pixel (all pixels if pix is None)."""
    pk = _Pack(scene, views, settings)
    if depth32 is None:
        depth32 = project32(scene, views, settings)["depth"]
    depth32 = np.ascontiguousarray(depth32, dtype=np.float32)
    pix, m = _pix(views, pix)
    fm = None if flip_masks is None else np.ascontiguousarray(flip_masks, dtype=np.uint32)
    img = np.zeros(m, np.float64)
    tf = np.zeros(m, np.float64)
    last = np.zeros(m, np.int32)
    cnt = np.zeros(m, np.int32)
    flags = np.zeros(m, np.int32)
    nflag = np.zeros(m, np.int32)
    rc = lib().or_render(C.byref(pk.scene), C.byref(pk.views), C.byref(pk.cfg), _p(depth32),
                         m, _p(pix), _p(fm), _p(img), _p(tf), _p(last), _p(cnt), _p(flags),
                         _p(nflag), threads)
    if rc:
        raise RuntimeError(f"or_render failed ({rc})")
    out = dict(image=img, t_final=tf, last_id=last, n_contrib=cnt, flags=flags, n_flagged=nflag)
    if pix is None:
        shp = (views.n_views, views.height, views.width)
        out = {k: v.reshape(shp) for k, v in out.items()}
    return out


def render_alternatives(scene, views, settings, pix, n_flagged, max_flags=3,
                        depth32=None, threads=0):
    """Every outcome of flipping the first min(n_flagged, max_flags) flagged
    decisions of each listed pixel. Returns arrays [n_pix, 2^max_flags] (NaN /
    -2 where a mask is beyond that pixel's count)."""
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    n_flagged = np.asarray(n_flagged)
    A = 1 << max_flags
    rep = np.repeat(pix, A, axis=0)
    masks = np.tile(np.arange(A, dtype=np.uint32), pix.shape[0])
    r = render(scene, views, settings, rep, masks, depth32, threads)
    img = r["image"].reshape(-1, A).copy()
    tf = r["t_final"].reshape(-1, A).copy()
    last = r["last_id"].reshape(-1, A).copy()
    valid = np.arange(A)[None, :] < (1 << np.minimum(n_flagged, max_flags))[:, None]
    img[~valid] = np.nan
    tf[~valid] = np.nan
    last[~valid] = -2
    return dict(image=img, t_final=tf, last_id=last)


def render_backward(scene, views, settings, dL_dC, pix=None, depth32=None, threads=0,
                    want_2d=False, flip_masks=None):
    """FP64 gradient of sum_p dL_dC[p] C(p) with respect to every input.

    flip_masks (per requested pixel, optional) differentiates each pixel along
    the forward walk with those flagged decisions inverted (see render)."""
    pk = _Pack(scene, views, settings)
    if depth32 is None:
        depth32 = project32(scene, views, settings)["depth"]
    depth32 = np.ascontiguousarray(depth32, dtype=np.float32)
    pix, m = _pix(views, pix)
    g = np.ascontiguousarray(np.asarray(dL_dC, dtype=np.float64).reshape(-1))
    assert g.size == m
    fm = None if flip_masks is None else np.ascontiguousarray(
        np.asarray(flip_masks, dtype=np.uint32).reshape(-1))
    assert fm is None or fm.size == m
    n, k, V = scene.n, scene.feat.shape[1], views.n_views
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n), feat=np.zeros((n, k)), b_iso=np.zeros(k),
               B_dir=np.zeros(np.asarray(scene.B_dir).shape), pose=np.zeros((V, 3, 4)))
    kl = int(np.asarray(scene.B_dir).shape[0])
    g2 = np.zeros((V, n, 7 + kl)) if want_2d else None
    rc = lib().or_render_backward(
        C.byref(pk.scene), C.byref(pk.views), C.byref(pk.cfg), _p(depth32), m, _p(pix), _p(fm), _p(g),
        _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logits"]),
        _p(out["feat"]), _p(out["b_iso"]), _p(out["B_dir"]), _p(out["pose"]), _p(g2), threads)
    if rc:
        raise RuntimeError(f"or_render_backward failed ({rc})")
    if want_2d:
        out["grad2d"] = g2
    return out


def count_inside(scene, views, settings, pix=None, depth32=None, threads=0):
    """Per pixel: Gaussians with q <= q_max at the pixel centre (whole list)."""
    pk = _Pack(scene, views, settings)
    if depth32 is None:
        depth32 = project32(scene, views, settings)["depth"]
    depth32 = np.ascontiguousarray(depth32, dtype=np.float32)
    pix, m = _pix(views, pix)
    out = np.zeros(m, np.int32)
    rc = lib().or_count_inside(C.byref(pk.scene), C.byref(pk.views), C.byref(pk.cfg),
                               _p(depth32), m, _p(pix), _p(out), threads)
    if rc:
        raise RuntimeError(f"or_count_inside failed ({rc})")
    return out if pix is not None else out.reshape(views.n_views, views.height, views.width)
