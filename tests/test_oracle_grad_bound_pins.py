"""Pins of the oracle's per-element bounds on the refit gradients.

oracle.color_grad_bound bounds how far a float32 blend's colour gradient
dL/dc_i = sum_p dL/dy_p alpha_i(p) T_i(p) (Sec. 3.3, Eq. 6-7 restricted to
the colours) may lie from the FP64 oracle's, and oracle.sh_grad_bound
carries it through Eq. 2 and the clamp of the shown colour. The bounds are
pinned against a float32 implementation of the same walk (other summation
order, float32 alpha and T) on a small workload, and on hand-made decisions
in doubt (a stop at T = 1e-4, alpha at 1/255, two splats at one depth, a
colour clamped at exactly 0), where the float32 side may take either branch
and the bound must hold the whole term.
"""
import math

import numpy as np

import oracle
from paper_2511_18441_b300 import scenegen as sg

Y00 = 0.5 / math.sqrt(math.pi)
CAM = sg.axis_camera(17, 17, 60.0, 2.0)   # pixel (8, 8) sits on the optical axis


def stack(zs, logits, rgbs, scale=0.05):
    """On-axis isotropic splats at depths zs showing colour rgb (DC only)."""
    n = len(zs)
    sh = np.zeros((16, 3, n))
    sh[0] = (np.asarray(rgbs, np.float64).T - 0.5) / Y00
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return sg.Scene(f(np.stack([np.zeros(n), np.zeros(n), np.asarray(zs, np.float64)])),
                    f(np.full((3, n), math.log(scale))), f(np.tile([[1.0], [0], [0], [0]], n)),
                    f(logits), f(sh))


def logit(p):
    return math.log(p / (1 - p))


def frame(scene, cam, seed=0):
    """Render, an L1 gradient against a target 0.02-0.1 away from it, and
    the oracle's colour gradient with its bound."""
    ref, sp, order, off, ids = oracle.render_image(scene, cam)
    rng = np.random.default_rng(seed)
    y = ref["rgb"]
    target = y + rng.choice([-1.0, 1.0], size=y.shape) * rng.uniform(0.02, 0.1, size=y.shape)
    _, g = oracle.l1_loss_grad(y, target)
    gr = oracle.color_grad(sp, off, ids, g)
    b = oracle.color_grad_bound(sp, off, ids, g)
    return sp, off, ids, g, gr, b


def f32_color_grad(sp, off, ids, g, width, height):
    """The colour gradient of a float32 walk: the oracle's splats rounded to
    float32, alpha = min(0.99, sigma exp(p)) with p in float32, skip below
    1/255, stop before T (1 - alpha) < 1e-4, products and the per-splat sums
    (pixels in tile order) in float32."""
    f32 = np.float32
    n = sp["n"]
    u, v = sp["u"].astype(f32), sp["v"].astype(f32)
    A, B, Cc = (sp["conic"][k::3].astype(f32) for k in range(3))
    sig = sp["opacity"].astype(f32)
    valid = sp["valid"].astype(bool)
    out = np.zeros((n, 3), f32)
    g32 = np.asarray(g, f32).reshape(height, width, 3)
    tx = (width + 15) // 16
    for t in range(len(off) - 1):
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        xs, ys = np.meshgrid(np.arange(x0, min(x0 + 16, width)), np.arange(y0, min(y0 + 16, height)))
        xs, ys = xs.ravel().astype(f32), ys.ravel().astype(f32)
        gp = g32[ys.astype(int), xs.astype(int)]
        T = np.ones(len(xs), f32)
        live = np.ones(len(xs), bool)
        for k in range(off[t], off[t + 1]):
            i = int(ids[k])
            if not valid[i]:
                continue
            dx, dy = xs - u[i], ys - v[i]
            p = (f32(-0.5) * (A[i] * dx * dx + Cc[i] * dy * dy) - B[i] * dx * dy).astype(f32)
            p = np.minimum(p, f32(0))
            al = np.minimum(f32(0.99), (sig[i] * np.exp(p)).astype(f32))
            take = live & (al >= f32(1.0 / 255.0))
            nT = (T * (f32(1) - al)).astype(f32)
            stop = take & (nT < f32(1e-4))
            live &= ~stop
            take &= ~stop
            w = np.where(take, (al * T).astype(f32), f32(0))
            for ch in range(3):
                for val in (gp[take, ch] * w[take]).astype(f32):
                    out[i, ch] = f32(out[i, ch] + val)
            T = np.where(take, nT, T)
    return out.astype(np.float64)


def test_color_grad_bound_covers_a_float32_walk():
    """Small workload: every element of the float32 walk's gradient within
    the bound; the bound well below the gradients it bounds."""
    w = sg.tiny_workload(n=1500, width=64, height=48)
    sp, off, ids, g, gr, b = frame(w.scene, w.camera, seed=3)
    g32 = f32_color_grad(sp, off, ids, g, 64, 48)
    err = np.abs(g32 - gr)
    assert np.all(err <= b), (err / np.maximum(b, 1e-300)).max()
    nz = np.abs(gr) > 0
    assert nz.sum() > 500
    assert np.median(b[nz] / np.abs(gr[nz])) < 1e-2


def test_a_stop_in_doubt_counts_the_whole_term():
    """Three opaque splats (alpha 0.99): after two, T = 1e-4 up to rounding.
    The second splat's term alpha T (1 - alpha) |g| may be present or not."""
    sc = stack([0.0, 0.05, 0.1], [logit(0.995)] * 3, [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1),
                                                      (0.1, 0.1, 0.9)])
    sp, off, ids, g, gr, b = frame(sc, CAM)
    gpix = np.abs(g[8, 8])
    a = 0.99
    assert np.all(b[1] >= gpix * a * (1 - a) * (1 - 1e-9))
    # the first splat's term is certain: only rounding-sized
    assert np.all(b[0] <= 1e-3 * np.abs(gr[0]))


def test_alpha_at_the_cutoff_counts_the_whole_term():
    """alpha three pixels from the centre is 1/255 up to rounding: at pixel
    (11, 8) the splat may be taken or skipped."""
    sigma = 0.5
    v = 9.0 / (2.0 * math.log(255 * sigma))
    s = 2.0 * math.sqrt(v - 0.3) / CAM.fy
    sc = stack([0.0], [logit(sigma)], [(0.3, 0.6, 0.9)], scale=s)
    sp, off, ids, g, gr, b = frame(sc, CAM)
    var = sp["cov2d"][0]
    a = sp["opacity"][0] * math.exp(-9.0 / (2.0 * var))
    assert abs(a * 255 - 1) < 1e-5
    assert np.all(b[0] >= np.abs(g[8, 11]) * a * (1 - 1e-6))


def test_two_splats_at_one_depth_may_swap():
    """Equal depths: either may be first, so each one's T may carry the
    other's factor (1 - alpha); the bound holds the difference."""
    sc = stack([0.1, 0.1], [logit(0.5), logit(0.25)], [(0.9, 0.1, 0.1), (0.1, 0.2, 0.8)])
    sp, off, ids, g, gr, b = frame(sc, CAM)
    aa, ab = sp["opacity"]
    gpix = np.abs(g[8, 8])
    # first as walked (index order): T = 1; swapped: T = 1 - ab
    assert np.all(b[0] >= gpix * aa * ab * (1 - 1e-9))
    # second: T = 1 - aa as walked, 1 if swapped
    assert np.all(b[1] >= gpix * ab * aa * (1 - 1e-9))


def test_distinct_depths_leave_only_rounding():
    """No decision in doubt: with dL/dy of one sign (no cancellation in
    the sums) the bound is a small fraction of the gradient."""
    sc = stack([0.1, 0.101], [logit(0.5), logit(0.25)], [(0.9, 0.1, 0.1), (0.1, 0.2, 0.8)])
    sp, off, ids, g, gr, b = frame(sc, CAM)
    gp = np.abs(g)
    assert np.all(oracle.color_grad_bound(sp, off, ids, gp) <= 1e-3 * oracle.color_grad(sp, off, ids, gp))


def test_sh_grad_bound_and_the_clamp():
    """Eq. 2 chained: the bound holds a float32 Y_k(d) g product; a colour
    clamped at exactly 0 may pass the gradient or not (the whole value), a
    colour far below 0 passes nothing on either side."""
    sc = stack([0.0, 0.05, 0.1], [logit(0.5)] * 3, [(0.6, 0.0, 0.4), (0.3, 0.7, -0.4),
                                                   (0.5, 0.5, 0.5)])
    sp, off, ids, g, gr, b = frame(sc, CAM)
    gs = oracle.sh_grad(sc, sp, gr)
    bs = oracle.sh_grad_bound(sc, sp, gr, b)
    # splat 0 green: f + 0.5 = 0 (in doubt); splat 1 blue: clamped for sure
    assert np.all(bs[:, 1, 0] >= np.abs(gs[:, 1, 0]))
    assert bs[0, 1, 0] >= Y00 * abs(gr[0, 1]) * (1 - 1e-9)
    assert np.all(gs[:, 2, 1] == 0) and np.all(bs[:, 2, 1] == 0)
    # a float32 Y_k(d) g (the direction is the optical axis: only the
    # z-harmonics are nonzero) lies within the bound
    d = np.float32([0.0, 0.0, 1.0])
    Y = np.zeros(16, np.float32)
    Y[0] = np.float32(0.28209479177387814)
    Y[2] = np.float32(0.4886025119029199) * d[2]
    Y[6] = np.float32(0.31539156525252005) * (np.float32(3) * d[2] * d[2] - np.float32(1))
    Y[12] = np.float32(0.3731763325901154) * d[2] * (np.float32(5) * d[2] * d[2] - np.float32(3))
    for i in (0, 2):
        for ch in range(3):
            if sp["rgb"][3 * i + ch] <= 0:
                continue
            g32 = (Y * np.float32(gr[i, ch])).astype(np.float64)
            assert np.all(np.abs(g32 - gs[:, ch, i]) <= bs[:, ch, i])
