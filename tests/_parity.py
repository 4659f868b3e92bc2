"""Helpers that compare the CUDA library's outputs with the CPU oracle.

Tolerances (stated once, used by every GPU parity test):
  binning (tiles touched, sorted keys and values, ranges): bit-exact;
  image and final transmittance: max |gpu - oracle| <= 1e-4 * (image range);
  gradients: per group ||g_gpu - g_or||_2 <= 1e-3 ||g_or||_2 and
             max |g_gpu - g_or| <= 1e-3 max |g_or|.
A pixel whose oracle walk met a decision within the window of a cutoff may
legitimately differ; it passes if it matches one of the oracle's outcomes with
those decisions flipped (at most 3 flagged decisions enumerated).
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


def check_image(scene, views, st, img, tf, ids=None, depth32=None, pix=None):
    """Compare a GPU render with the oracle; returns a small report dict.

    img, tf, ids are [V,H,W] arrays (or [M] when pix lists the pixels)."""
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
    cand = ~ok & flagged
    unresolved = 0
    if cand.any():
        if pix is None:
            V, H, W = img.shape
            vv, rr, cc = np.nonzero(cand)
            plist = np.stack([vv, rr, cc], 1)
        else:
            plist = pix[cand]
        nf = ref["n_flagged"][cand]
        alt = oracle.render_alternatives(scene, views, st, plist, nf, depth32=depth32)
        gi, gt_, gid = img[cand], tf[cand], None if ids is None else ids[cand]
        match = (np.abs(alt["image"] - gi[:, None]) <= tol) & (np.abs(alt["t_final"] - gt_[:, None]) <= tol)
        if gid is not None:
            match &= alt["last_id"] == gid[:, None]
        resolved = match.any(axis=1)
        unresolved = int((~resolved & (nf > 3)).sum())
        assert (resolved | (nf > 3)).all(), (
            f"{int((~resolved & (nf <= 3)).sum())} flagged pixels match no outcome")
    n = img.size
    return dict(range=rng, max_err=float(np.abs(img - rimg).max()) if n else 0.0,
                flagged_frac=float(flagged.mean()) if n else 0.0,
                unresolved_frac=unresolved / max(n, 1), ref=ref)


def compare_grads(gpu: dict, ref: dict, names, tol=GRAD_TOL):
    out = {}
    for n in names:
        a = np.asarray(gpu[n], np.float64).reshape(-1)
        b = np.asarray(ref[n], np.float64).reshape(-1)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.abs(a).max(initial=0) == 0, n
            continue
        rel = np.linalg.norm(a - b) / nb
        mx = np.abs(a - b).max() / np.abs(b).max()
        out[n] = (rel, mx)
        assert rel <= tol and mx <= tol, (n, rel, mx)
    return out
