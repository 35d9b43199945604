"""Shared comparison logic for the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (FP32 path): images within max-abs 2e-4 per RGB channel on
pixels the oracle does not flag; masks and tile lists bit-exact except for
flagged Gaussians, with Gaussians whose FP64 depths agree to 1e-6 relative
allowed to swap places (their float32 depth keys may tie or cross).
"""
import numpy as np

IMAGE_TOL = 2e-4
DEPTH_REL = 1e-6


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


def check_image(gpu_rgb, gpu_T, ref, pixels=None, tol=IMAGE_TOL, max_flag_frac=0.02):
    """gpu_rgb (H,W,3), gpu_T (H,W) numpy; ref: oracle dict with full-size
    arrays; pixels: optional boolean (H,W) mask of pixels to compare."""
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
                max_err_flagged=float(err[sel & flag].max()) if n_flag else 0.0)
    if worst > tol or worstT > tol:
        y, x = np.unravel_index(np.argmax(np.where(use, err, -1)), err.shape)
        raise AssertionError(f"image mismatch {info}; worst pixel ({x},{y}) gpu "
                             f"{gpu_rgb[y, x]} ref {ref['rgb'][y, x]}")
    assert n_flag <= max_flag_frac * max(n_sel, 1), f"too many flagged pixels {info}"
    return info


def check_tile_lists(gpu_ranges, gpu_ids, sp, off, ids, tiles=None):
    """Per tile, the GPU list equals the oracle's after dropping flagged
    Gaussians, up to swaps of Gaussians with FP64 depths within 1e-6."""
    flagged = sp["fp_flag"] > 0
    depth = sp["depth"]
    n_tiles = len(off) - 1
    tiles = range(n_tiles) if tiles is None else tiles
    checked = 0
    for t in tiles:
        g = gpu_ids[gpu_ranges[t, 0]:gpu_ranges[t, 1]].astype(np.int64)
        o = ids[off[t]:off[t + 1]].astype(np.int64)
        g = g[~flagged[g]]
        o = o[~flagged[o]]
        if np.array_equal(g, o):
            checked += len(g)
            continue
        assert len(g) == len(o) and np.array_equal(np.sort(g), np.sort(o)), \
            f"tile {t}: different Gaussians ({len(g)} vs {len(o)})"
        z = depth[g]
        dz = np.diff(z)
        tol = DEPTH_REL * np.abs(z[1:])
        assert np.all(dz >= -tol), f"tile {t}: out of depth order beyond 1e-6"
        checked += len(g)
    return checked
