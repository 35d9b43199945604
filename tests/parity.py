"""Shared comparison logic for the GPU parity tests (CUDA path vs FP64 oracle).

Images (FP32 path): every pixel the oracle does not flag within max-abs 2e-4
per RGB channel (and T); every flagged pixel (a decision float32 may take the
other way: alpha near 1/255, T near the 1e-4 stop, a selection near the
region's boundary, two contributors whose float32 depth keys may be equal)
within 2e-4 of one of the outcomes those decisions allow, each evaluated by
the oracle in FP64. Flagged pixels are expected to stay below MAX_FLAG_FRAC
of the frame: the largest observed fractions are 0.42% at 3M Gaussians and
1920x1080 and 0.68% on 1280x720 views of a 4M scene, where the stop decision
after hundreds of contributors per pixel dominates.

Tile lists: bit-exact. Each GPU depth key is the float32 the oracle rounds
the FP64 depth to (either neighbour where the depth lies within 1e-12 of a
rounding midpoint), and each tile's list is the oracle's set of Gaussians in
(key, index) order: the (depth, index) order of Eq. 3 except that Gaussians
with equal float32 keys are ordered by index. Gaussians whose tile range or
visibility the oracle flags may be present or absent.
"""
import numpy as np

import oracle

IMAGE_TOL = 2e-4
MAX_FLAG_FRAC = 0.01


def to_np(t):
    return t.detach().cpu().numpy()


def check_mask(gpu_mask_words, n, ref_sel, ref_flag):
    bits = np.unpackbits(gpu_mask_words.view(np.uint8), bitorder="little")[:n]
    pad = np.unpackbits(gpu_mask_words.view(np.uint8), bitorder="little")[n:]
    assert not pad.any(), "padding bits of the mask must be zero"
    ok = ref_flag == 0
    bad = np.flatnonzero(ok & (bits != ref_sel))
    assert bad.size == 0, f"{bad.size} unflagged mask bits differ, e.g. {bad[:10]}"
    return bits


def flagged_outcome_errors(gpu_rgb, gpu_T, sp, off, ids, xs, ys, bg=(0.0, 0.0, 0.0)):
    """Per listed pixel: the smallest max-abs distance of the GPU's (r, g, b,
    T) to an outcome the oracle allows there, and the number of outcomes."""
    out, cnt = oracle.pixel_outcomes(sp, off, ids, xs, ys, bg=bg)
    over = np.flatnonzero(cnt < 0)
    for j in over:   # rare: many decisions in doubt at one pixel
        o1, c1 = oracle.pixel_outcomes(sp, off, ids, xs[j:j + 1], ys[j:j + 1], bg=bg,
                                       max_out=1 << 16)
        assert c1[0] >= 0, f"pixel ({xs[j]}, {ys[j]}): more than 65536 outcomes"
        best = np.abs(o1[0, :c1[0]] - np.append(gpu_rgb[ys[j], xs[j]], gpu_T[ys[j], xs[j]])).max(-1)
        out[j, 0] = o1[0, np.argmin(best)]
        cnt[j] = 1
    g = np.concatenate([gpu_rgb[ys, xs], gpu_T[ys, xs][:, None]], 1)
    d = np.abs(out - g[:, None, :]).max(-1)
    d = np.where(np.arange(out.shape[1])[None, :] < cnt[:, None], d, np.inf)
    return d.min(1), cnt


def check_image(gpu_rgb, gpu_T, ref, sp=None, off=None, ids=None, bg=(0.0, 0.0, 0.0),
                pixels=None, tol=IMAGE_TOL, max_flag_frac=MAX_FLAG_FRAC):
    """gpu_rgb (H,W,3), gpu_T (H,W) numpy; ref: the oracle's image dict;
    sp, off, ids: its splats and tile lists (needed to check the flagged
    pixels); pixels: optional boolean (H,W) mask of pixels to compare."""
    H, W = gpu_T.shape
    sel = np.ones((H, W), bool) if pixels is None else pixels
    flag = ref["flag"] > 0
    err = np.abs(gpu_rgb - ref["rgb"]).max(-1)
    errT = np.abs(gpu_T - ref["T"])
    use = sel & ~flag
    n_sel = int(sel.sum())
    n_flag = int((sel & flag).sum())
    worst = float(err[use].max()) if use.any() else 0.0
    worstT = float(errT[use].max()) if use.any() else 0.0
    info = dict(pixels=n_sel, flagged=n_flag, max_err=worst, max_err_T=worstT,
                max_err_flagged_vs_fp64_path=float(err[sel & flag].max()) if n_flag else 0.0)
    if worst > tol or worstT > tol:
        y, x = np.unravel_index(np.argmax(np.where(use, err, -1)), err.shape)
        raise AssertionError(f"image mismatch {info}; worst pixel ({x},{y}) gpu "
                             f"{gpu_rgb[y, x]} ref {ref['rgb'][y, x]}")
    if n_flag:
        assert sp is not None, "flagged pixels need the oracle's splats and tile lists"
        ys, xs = np.nonzero(sel & flag)
        best, cnt = flagged_outcome_errors(gpu_rgb, gpu_T, sp, off, ids, xs, ys, bg)
        info["max_err_flagged_best_outcome"] = float(best.max())
        info["max_outcomes_per_flagged_pixel"] = int(cnt.max())
        if best.max() > tol:
            j = int(np.argmax(best))
            raise AssertionError(f"flagged pixel ({xs[j]},{ys[j]}) matches none of its "
                                 f"{cnt[j]} outcomes (closest {best[j]:.3g}) {info}")
    assert n_flag <= max_flag_frac * max(n_sel, 1), f"too many flagged pixels {info}"
    return info


def check_tile_lists(gpu_ranges, gpu_ids, gpu_keys, sp, off, ids, tiles=None):
    """Per tile, the GPU list equals the oracle's Gaussians in (GPU key,
    index) order (Gaussians with a flagged tile range or visibility dropped
    from both), and every GPU key of a listed Gaussian is a float32 rounding
    of its FP64 depth: the nearest, or either neighbour where the depth lies
    within 1e-12 of a midpoint. Returns the number of pairs checked."""
    flagged = sp["fp_flag"] > 0
    k32, amb = oracle.depth_keys(sp)
    keys = np.asarray(gpu_keys, np.float32)
    vis = (sp["visible"] > 0) & ~flagged
    exact = vis & ~amb
    bad = np.flatnonzero(exact & (keys != k32))
    assert bad.size == 0, f"{bad.size} depth keys differ from the float32 nearest the depth, " \
                          f"e.g. {bad[:5]}: {keys[bad[:5]]} vs {k32[bad[:5]]}"
    d = np.asarray(sp["depth"], np.float64)
    up = np.nextafter(k32, np.float32(np.inf))
    dn = np.nextafter(k32, np.float32(-np.inf))
    other = np.where(k32.astype(np.float64) <= d, up, dn)
    bad = np.flatnonzero(vis & amb & (keys != k32) & (keys != other))
    assert bad.size == 0, f"{bad.size} depth keys near a rounding midpoint take neither float32"
    n_tiles = len(off) - 1
    tiles = range(n_tiles) if tiles is None else tiles
    checked = 0
    for t in tiles:
        g = gpu_ids[gpu_ranges[t, 0]:gpu_ranges[t, 1]].astype(np.int64)
        o = ids[off[t]:off[t + 1]].astype(np.int64)
        g = g[~flagged[g]]
        o = o[~flagged[o]]
        o = o[np.lexsort((o, keys[o]))]
        if not np.array_equal(g, o):
            assert len(g) == len(o) and np.array_equal(np.sort(g), np.sort(o)), \
                f"tile {t}: different Gaussians ({len(g)} vs {len(o)})"
            k = int(np.flatnonzero(g != o)[0])
            raise AssertionError(f"tile {t}: position {k} holds {g[k]} (key {keys[g[k]]!r}), "
                                 f"(key, index) order wants {o[k]} (key {keys[o[k]]!r})")
        checked += len(g)
    return checked
