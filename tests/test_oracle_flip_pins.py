"""Pins of the oracle's near-cutoff enumeration (no GPU).

Eq. 1 is applied with three cutoffs (the S4 reading: a Gaussian is skipped
when q > q_max or sigma < alpha_min, and the walk stops before adding one
whose T' would fall below t_min). A binary32 renderer can take any of these
decisions the other way when the FP64 value sits very close to the cutoff, so
the oracle numbers every decision met within a window of its cutoff and bit d
of a flip mask inverts the d-th one. The GPU parity tests accept a flagged
pixel when it matches one of those outcomes, and differentiate it along the
matched one.

These tests build one-pixel scenes with exactly the decisions they need, each
placed just inside its window, and check every mask against
  * the Eq. 1 sum C = sum_j c_j sigma_j prod_{l<j} (1 - sigma_l) written out by
    hand for the Gaussians that mask keeps, and
  * the plain walk (mask 0) under a cutoff moved to the other side of the
    value, which takes the inverted decision without any mask; the forward
    outputs must agree exactly, the backward up to summation order.
A numbering slip (bit d flipping another decision), an inverted sense, or a
flip that leaks into a later decision fails one of them.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2406_02518_gb300 import synthetic as syn

SDD, SID, PITCH = 4.0, 2.0, 1.0 / 16.0  # 64 px per world unit at the isocentre
ISO_LOG_SCALE = math.log(0.05)           # 1.6 px footprint at the isocentre
GROUPS = ["means", "log_scales", "quats", "opacity_logits", "feat", "b_iso", "B_dir", "pose"]


def _logit(p):
    return math.log(p / (1.0 - p))


def _sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def _view():
    pose = syn.pose_matrix(np.eye(3), np.array([0.0, 0.0, SID]))[None].astype(np.float32)
    return syn.Views(np.ascontiguousarray(pose), syn.detector(1, SDD, PITCH), 1, 1)


def _scene(gs):
    """gs: list of (x, z, alpha); every Gaussian isotropic, on the row y = 0 of
    the single pixel (whose centre is on the optical axis)."""
    n = len(gs)
    means = np.array([[x, 0.0, z] for x, z, _ in gs], np.float32)
    log_s = np.full((n, 3), ISO_LOG_SCALE, np.float32)
    quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1))
    logits = np.array([_logit(a) for _, _, a in gs], np.float32)
    rng = np.random.default_rng(7)
    feat = rng.uniform(-1.0, 1.0, (n, 8)).astype(np.float32)
    b_iso = rng.uniform(-1.0, 1.0, 8).astype(np.float32)
    return syn.Scene(means, log_s, quats, logits, feat, n, b_iso, np.zeros((3, 8), np.float32))


def _settings(**kw):
    return dataclasses.replace(syn.Settings(near_plane=0.2, dilation=0.0), **kw)


def _q_at_pixel(scene, views, st, i):
    """q of Gaussian i at the pixel centre, from the (separately pinned) projection."""
    P = oracle.project64(scene, views, st)[0, i]
    dx, dy = P[0] - 0.5, P[1] - 0.5
    return P[2] * dx * dx + 2 * P[3] * dx * dy + P[4] * dy * dy


def _place_q(gs, i, q_target, st):
    """Move Gaussian i along x until its q at the pixel is q_target."""
    gs = list(gs)
    views = _view()
    for _ in range(6):
        q = _q_at_pixel(_scene(gs), views, st, i)
        x, z, a = gs[i]
        gs[i] = (float(np.float32(x * math.sqrt(q_target / q))), z, a)
    return gs


def _terms(scene, views, st):
    """sigma_j and c_j of every Gaussian at the pixel, written from Eq. 1 and
    Eq. 3 (c = sigmoid(b_iso . f) for an isotropic Gaussian), in FP64."""
    sig, col, q = [], [], []
    for i in range(scene.n):
        qi = _q_at_pixel(scene, views, st, i)
        a = _sigmoid(float(scene.opacity_logits[i]))
        sig.append(min(st.alpha_max, a * math.exp(-0.5 * qi)))
        col.append(_sigmoid(float(np.dot(scene.b_iso.astype(np.float64), scene.feat[i].astype(np.float64)))))
        q.append(qi)
    return np.array(sig), np.array(col), np.array(q)


def _eq1(sig, col, kept):
    """Eq. 1 over the kept Gaussians in depth order (the list order here)."""
    C, T, last = 0.0, 1.0, -1
    for j in kept:
        C += col[j] * sig[j] * T
        T *= 1.0 - sig[j]
        last = j
    return C, T, last


PIX = np.array([[0, 0, 0]], np.int32)


def _check_masks(scene, st, expect, moved):
    """expect[m] = the kept Gaussians under mask m; moved[m] = settings whose
    plain walk takes mask m's decisions (None: not checked that way)."""
    views = _view()
    sig, col, _ = _terms(scene, views, st)
    nf = int(math.log2(len(expect)))
    plain = oracle.render(scene, views, st)
    assert int(plain["n_flagged"][0, 0, 0]) == nf
    alt = oracle.render_alternatives(scene, views, st, PIX, np.array([nf]))
    for m, kept in enumerate(expect):
        C, T, last = _eq1(sig, col, kept)
        assert abs(alt["image"][0, m] - C) < 1e-14, (m, alt["image"][0, m], C)
        assert abs(alt["t_final"][0, m] - T) < 1e-14, (m, alt["t_final"][0, m], T)
        assert alt["last_id"][0, m] == last, (m, alt["last_id"][0, m], last)
    # masks past the pixel's decisions are marked absent
    assert np.isnan(alt["image"][0, len(expect):]).all()
    assert (alt["last_id"][0, len(expect):] == -2).all()
    # mask 0 is the plain walk
    assert alt["image"][0, 0] == plain["image"][0, 0, 0]
    assert alt["last_id"][0, 0] == plain["last_id"][0, 0, 0]
    # every mask equals the plain walk under a cutoff moved past the value,
    # forward and backward
    w = np.ones(1)
    for m, st_m in enumerate(moved):
        if st_m is None:
            continue
        r = oracle.render(scene, views, st_m, pix=PIX)
        fl = oracle.render(scene, views, st, pix=PIX, flip_masks=np.array([m], np.uint32))
        assert fl["image"][0] == r["image"][0] and fl["t_final"][0] == r["t_final"][0]
        assert fl["last_id"][0] == r["last_id"][0]
        g_flip = oracle.render_backward(scene, views, st, w, pix=PIX,
                                        flip_masks=np.array([m], np.uint32))
        g_move = oracle.render_backward(scene, views, st_m, w, pix=PIX)
        for k in GROUPS:  # equal up to the order of the oracle's threaded sums
            np.testing.assert_allclose(g_flip[k], g_move[k], rtol=1e-12, atol=1e-15,
                                       err_msg=f"mask {m} {k}")
    # and the masked backward differs from the plain one wherever the kept set does
    g0 = oracle.render_backward(scene, views, st, w, pix=PIX)
    for m in range(1, len(expect)):
        if sorted(expect[m]) != sorted(expect[0]):
            gm = oracle.render_backward(scene, views, st, w, pix=PIX,
                                        flip_masks=np.array([m], np.uint32))
            assert np.abs(gm["opacity_logits"] - g0["opacity_logits"]).max() > 1e-6


@pytest.mark.parametrize("side", [-1, 1])
def test_flip_of_the_q_cutoff(side):
    """F in front (sigma 0.5) and A behind it with q = 9 -/+ 1e-4: A is kept
    (side -1) or skipped (side +1) by the plain walk; mask 1 does the other."""
    st = _settings()
    gs = _place_q([(0.0, -0.3, 0.5), (0.15, 0.0, 0.9)], 1, st.q_max + side * 1e-4, st)
    scene, views = _scene(gs), _view()
    sig, _, q = _terms(scene, views, st)
    assert abs(q[1] - (st.q_max + side * 1e-4)) < 1e-5
    assert sig[1] > 2 * st.alpha_min  # the decision matters (A would pass alpha_min)
    keep, drop = [0, 1], [0]
    expect = [keep, drop] if side < 0 else [drop, keep]
    other = _settings(q_max=st.q_max + side * 2e-4)  # the cutoff moved past q
    _check_masks(scene, st, expect, [None, other])


@pytest.mark.parametrize("side", [-1, 1])
def test_flip_of_the_alpha_min_cutoff(side):
    """B on the axis behind F with alpha = alpha_min (1 -/+ 3e-4) at G = 1."""
    st = _settings()
    scene = _scene([(0.0, -0.3, 0.5), (0.0, 0.1, st.alpha_min * (1 + side * 3e-4))])
    views = _view()
    sig, _, q = _terms(scene, views, st)
    assert q[1] == 0.0
    assert 1e-4 < side * (sig[1] / st.alpha_min - 1) < 1e-3
    keep, drop = [0, 1], [0]
    expect = [keep, drop] if side > 0 else [drop, keep]
    other = _settings(alpha_min=st.alpha_min * (1 + side * 6e-4))
    _check_masks(scene, st, expect, [None, other])


@pytest.mark.parametrize("side", [-1, 1])
def test_flip_of_the_t_min_stop(side):
    """Two Gaussians of sigma 0.95 leave T = 2.5e-3; the third one's T' is
    t_min (1 +/- 3e-5): the plain walk stops before it (side -1) or adds it."""
    st = _settings()
    a3 = 1.0 - 0.04 * (1 + side * 3e-5)
    scene = _scene([(0.0, -0.3, 0.95), (0.0, -0.2, 0.95), (0.0, 0.0, a3)])
    views = _view()
    sig, _, _ = _terms(scene, views, st)
    t_next = (1 - sig[0]) * (1 - sig[1]) * (1 - sig[2])
    assert 1e-5 < side * (t_next / st.t_min - 1) < 1e-4
    stop, go = [0, 1], [0, 1, 2]
    expect = [go, stop] if side > 0 else [stop, go]
    other = _settings(t_min=st.t_min * (1 + side * 6e-5))
    _check_masks(scene, st, expect, [None, other])


def test_two_decisions_are_numbered_in_the_order_met():
    """F (sigma 0.5), then A with q = 9 - 1e-4 (kept; decision 0), then B on
    the axis with sigma = alpha_min (1 - 3e-4) (skipped; decision 1).
    Bit 0 flips A, bit 1 flips B; mask 3 flips both."""
    st = _settings()
    gs = _place_q([(0.0, -0.3, 0.5), (0.15, 0.0, 0.9), (0.0, 0.1, st.alpha_min * (1 - 3e-4))],
                  1, st.q_max - 1e-4, st)
    scene, views = _scene(gs), _view()
    sig, _, q = _terms(scene, views, st)
    assert abs(q[1] - (st.q_max - 1e-4)) < 1e-5 and q[2] == 0.0
    expect = [[0, 1], [0], [0, 1, 2], [0, 2]]
    both = _settings(q_max=st.q_max - 2e-4, alpha_min=st.alpha_min * (1 - 6e-4))
    moved = [None,
             _settings(q_max=st.q_max - 2e-4),
             _settings(alpha_min=st.alpha_min * (1 - 6e-4)),
             both]
    _check_masks(scene, st, expect, moved)


def test_decisions_outside_the_windows_are_not_flagged():
    """The same scene with A at q = 8.9 and B at 1.01 alpha_min: no decision
    is numbered, and a mask changes nothing."""
    st = _settings()
    gs = _place_q([(0.0, -0.3, 0.5), (0.15, 0.0, 0.9), (0.0, 0.1, st.alpha_min * 1.01)],
                  1, 8.9, st)
    scene, views = _scene(gs), _view()
    plain = oracle.render(scene, views, st)
    assert plain["n_flagged"].max() == 0 and plain["flags"].max() == 0
    fl = oracle.render(scene, views, st, pix=PIX, flip_masks=np.array([7], np.uint32))
    assert fl["image"][0] == plain["image"][0, 0, 0]
