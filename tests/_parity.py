"""Helpers that compare the CUDA library's outputs with the CPU oracle.

Tolerances (stated once, used by every GPU parity test):
  binning (tiles touched, sorted keys and values, ranges): bit-exact;
  image and final transmittance: max |gpu - oracle| <= 1e-4 * (image range);
  gradients: per group ||g_gpu - g_or||_2 <= 1e-3 ||g_or||_2 and
             max |g_gpu - g_or| <= 1e-3 max |g_or|.
A pixel whose oracle walk met a decision within the window of a cutoff may
legitimately differ; it passes if it matches one of the oracle's outcomes with
those decisions flipped (at most 3 flagged decisions enumerated), and gradient
checks differentiate it along the outcome it matched. Pixels left unresolved
or out of a gradient check stay within 1e-3 of every view.
"""
import numpy as np

import oracle

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def compare_binning(gpu, ref):
    assert gpu["m"] == ref["m"], (gpu["m"], ref["m"])
    assert np.array_equal(gpu["tiles_touched"].reshape(ref["tiles_touched"].shape),
                          ref["tiles_touched"])
    assert np.array_equal(gpu["keys"], ref["keys"])
    assert np.array_equal(gpu["vals"], ref["vals"])
    assert np.array_equal(gpu["ranges"].reshape(ref["ranges"].shape), ref["ranges"])


def last_ids(n_last, bins, views, tile):
    """Map per-pixel tile-list positions to Gaussian ids (-1 when none)."""
    V, H, W = n_last.shape
    tx = -(-W // tile)
    tpv = tx * (-(-H // tile))
    rows, cols = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    gt = (np.arange(V)[:, None, None] * tpv + (rows // tile) * tx + cols // tile)
    start = bins["ranges"].reshape(-1, 2)[gt, 0].astype(np.int64)
    nl = n_last.astype(np.int64)
    ids = np.full(n_last.shape, -1, np.int64)
    has = nl > 0
    ids[has] = bins["vals"][start[has] + nl[has] - 1]
    return ids


# Oracle flags (oracle/ddgs_oracle.h) that no flip enumeration covers: the
# alpha_max clamp decides whether a gradient flows through alpha and G, and a
# depth at the near / far plane decides a whole Gaussian.
FLAG_NEAR_CLAMP, FLAG_NEAR_CULL = 4, 16
# Bounds on the pixels a comparison cannot use: flagged pixels (a decision in
# the window of a cutoff) are resolved against the enumerated outcomes; those
# still unresolved, and those the gradient check leaves out, stay below
# MASK_BOUND of the pixels of every view.
FLAG_BOUND = 0.05
MASK_BOUND = 1e-3


def _per_view(bad, pix):
    """Fraction of `bad` pixels in each view ([V,H,W] arrays, or lists with pix)."""
    if pix is None:
        return bad.reshape(bad.shape[0], -1).mean(axis=1)
    v = pix[:, 0]
    return np.array([bad[v == k].mean() for k in np.unique(v)])


def check_image(scene, views, st, img, tf, ids=None, depth32=None, pix=None):
    """Compare a GPU render with the oracle; returns a small report dict.

    img, tf, ids are [V,H,W] arrays (or [M] when pix lists the pixels).
    Every pixel is resolved to the oracle outcome the GPU took: mask 0 (the
    plain FP64 walk) for unflagged pixels; for a flagged pixel, among the
    outcomes with up to 3 flagged decisions inverted that match the GPU
    within the tolerance, the nearest one. report["masks"] holds the matched
    flip mask per pixel and report["unresolved"] marks flagged pixels that
    match none (only allowed past 3 flagged decisions)."""
    ref = oracle.render(scene, views, st, pix=pix, depth32=depth32)
    rimg = ref["image"]
    rng = float(rimg.max() - rimg.min()) if rimg.size else 0.0
    tol = IMG_TOL * max(rng, 1e-6)
    ok_img = np.abs(img - rimg) <= tol
    ok_tf = np.abs(tf - ref["t_final"]) <= tol
    ok_id = np.ones_like(ok_img) if ids is None else (ids == ref["last_id"])
    ok = ok_img & ok_tf & ok_id
    flagged = ref["n_flagged"] > 0
    plain_bad = ~ok & ~flagged
    assert not plain_bad.any(), (
        f"{plain_bad.sum()} unflagged pixels differ; max img err "
        f"{np.abs(img - rimg)[plain_bad].max():.3g} (tol {tol:.3g})")
    masks = np.zeros(img.shape, np.uint32)
    unresolved = np.zeros(img.shape, bool)
    if flagged.any():
        if pix is None:
            vv, rr, cc = np.nonzero(flagged)
            plist = np.stack([vv, rr, cc], 1)
        else:
            plist = pix[flagged]
        nf = ref["n_flagged"][flagged]
        alt = oracle.render_alternatives(scene, views, st, plist, nf, depth32=depth32)
        gi, gt_ = img[flagged], tf[flagged]
        d_img, d_tf = np.abs(alt["image"] - gi[:, None]), np.abs(alt["t_final"] - gt_[:, None])
        match = (d_img <= tol) & (d_tf <= tol)
        if ids is not None:
            match &= alt["last_id"] == ids[flagged][:, None]
        dist = np.where(match, np.maximum(d_img, d_tf), np.inf)
        resolved = match.any(axis=1)
        assert (resolved | (nf > 3)).all(), (
            f"{int((~resolved & (nf <= 3)).sum())} flagged pixels match no outcome")
        masks[flagged] = np.where(resolved, np.argmin(dist, axis=1), 0).astype(np.uint32)
        unresolved[flagged] = ~resolved
    n = img.size
    flagged_frac = float(flagged.mean()) if n else 0.0
    per_view_unres = _per_view(unresolved, pix) if n else np.zeros(1)
    assert flagged_frac <= FLAG_BOUND, f"{flagged_frac:.4f} of the pixels flagged"
    assert per_view_unres.max() <= MASK_BOUND, f"unresolved per view {per_view_unres}"
    return dict(range=rng, max_err=float(np.abs(img - rimg).max()) if n else 0.0,
                flagged_frac=flagged_frac, unresolved_frac=float(unresolved.mean()) if n else 0.0,
                masks=masks, unresolved=unresolved, pix=pix, ref=ref)


def gradient_weights(rep, seed):
    """dL/dC for a gradient check: U(-1, 1) on every pixel the image check
    resolved, 0 on the rest (unresolved flagged pixels and pixels near the
    alpha_max clamp or a culling plane). Returns (weights, flip masks); the
    oracle differentiates every pixel along its matched outcome. Asserts that
    the zeroed pixels stay within MASK_BOUND of every view, so that no check
    passes on an all-zero loss."""
    shape = rep["masks"].shape
    w = np.random.default_rng(seed).uniform(-1, 1, shape)
    drop = rep["unresolved"] | ((rep["ref"]["flags"] & (FLAG_NEAR_CLAMP | FLAG_NEAR_CULL)) != 0)
    per_view = _per_view(drop, rep["pix"]) if drop.size else np.zeros(1)
    assert per_view.max() <= MASK_BOUND, f"gradient check leaves out {per_view} of the pixels"
    rep["masked_frac"] = float(drop.mean()) if drop.size else 0.0
    return np.where(drop, 0.0, w), rep["masks"]


def compare_grads(gpu: dict, ref: dict, names, tol=GRAD_TOL, zero_ok=()):
    """Per group: relative L2 and max-abs errors within tol. A reference group
    that is exactly zero fails unless listed in zero_ok (then the GPU's must be
    zero too), so that a check cannot pass on an all-zero loss."""
    out = {}
    for n in names:
        a = np.asarray(gpu[n], np.float64).reshape(-1)
        b = np.asarray(ref[n], np.float64).reshape(-1)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert n in zero_ok, f"reference gradient of {n} is zero"
            assert np.abs(a).max(initial=0) == 0, n
            continue
        rel = np.linalg.norm(a - b) / nb
        mx = np.abs(a - b).max() / np.abs(b).max()
        out[n] = (rel, mx)
        assert rel <= tol and mx <= tol, (n, rel, mx)
    return out
