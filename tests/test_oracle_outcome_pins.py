"""Pins of the oracle's outcome enumeration for flagged pixels and of its
float32 depth keys.

A flagged pixel carries a decision of the walk of Eq. 3 (ReCoGS, arXiv
2511.18441, Sec. 3.1) that float32 arithmetic may take the other way. The
enumeration must return every outcome those decisions allow and nothing
else; each case below builds one such decision on hand-made splats centred
on a pixel (where G = 1 and alpha = sigma exactly) and checks the outcomes
against the closed-form composites of Eq. 3.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_18441_b300 import scenegen as sg

Y00 = 0.5 / math.sqrt(math.pi)


def stack(zs, logits, rgbs, scale=0.05, xs=None):
    """On-axis isotropic splats at depths zs (view-dependent terms zero, so
    each shows the colour rgb = Y00 C0 + 0.5)."""
    n = len(zs)
    xs = np.zeros(n) if xs is None else np.asarray(xs, np.float64)
    sh = np.zeros((16, 3, n))
    sh[0] = (np.asarray(rgbs, np.float64).T - 0.5) / Y00
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return sg.Scene(f(np.stack([xs, np.zeros(n), np.asarray(zs, np.float64)])),
                    f(np.full((3, n), math.log(scale))), f(np.tile([[1.0], [0], [0], [0]], n)),
                    f(logits), f(sh))


def frame(scene, cam, edit=None):
    ref, sp, order, off, ids = oracle.render_image(scene, cam, edit)
    return ref, sp, off, ids


def outcomes_at(sp, off, ids, x, y):
    out, cnt = oracle.pixel_outcomes(sp, off, ids, [x], [y])
    assert cnt[0] >= 1
    return out[0, :cnt[0]]


def same_set(got, want, tol=1e-12):
    got = np.asarray(got)
    want = np.asarray(want)
    assert len(got) == len(want), f"{len(got)} outcomes, expected {len(want)}: {got}"
    for w in want:
        assert np.abs(got - w).max(-1).min() <= tol, f"missing outcome {w} in {got}"


def logit(p):
    return math.log(p / (1 - p))


CAM = sg.axis_camera(17, 17, 60.0, 2.0)   # pixel (8, 8) sits on the optical axis


def test_equal_depth_pair_gives_both_orders():
    """Two splats at one depth (equal float32 keys, so a float32 sort orders
    them by index while the FP64 order may not be unique): both composites."""
    ca, cb = (0.9, 0.1, 0.1), (0.1, 0.2, 0.8)
    sc = stack([0.1, 0.1], [logit(0.5), logit(0.25)], [ca, cb])
    ref, sp, off, ids = frame(sc, CAM)
    assert ref["flag"][8, 8] & 16
    aa, ab = sp["opacity"]
    ca, cb = sp["rgb"][0:3], sp["rgb"][3:6]
    T = (1 - aa) * (1 - ab)
    same_set(outcomes_at(sp, off, ids, 8, 8),
             [np.append(ca * aa + cb * ab * (1 - aa), T),
              np.append(cb * ab + ca * aa * (1 - ab), T)])


def test_distinct_depths_give_one_order():
    """The same pair 1e-3 apart in depth (different keys): one outcome."""
    sc = stack([0.1, 0.101], [logit(0.5), logit(0.25)], [(0.9, 0.1, 0.1), (0.1, 0.2, 0.8)])
    ref, sp, off, ids = frame(sc, CAM)
    assert ref["flag"][8, 8] == 0
    aa, ab = sp["opacity"]
    ca, cb = sp["rgb"][0:3], sp["rgb"][3:6]
    same_set(outcomes_at(sp, off, ids, 8, 8),
             [np.append(ca * aa + cb * ab * (1 - aa), (1 - aa) * (1 - ab))])


def test_alpha_at_the_cutoff_gives_skip_and_take():
    """A splat whose alpha three pixels from its centre is 1/255 up to the
    float32 rounding of its scale: skipped (background, T = 1) or taken."""
    sigma = 0.5
    f, z = CAM.fy, 2.0
    v = 9.0 / (2.0 * math.log(255 * sigma))     # alpha(3 px) = sigma exp(-9 / (2 v)) = 1/255
    s = z * math.sqrt(v - 0.3) / f
    sc = stack([0.0], [logit(sigma)], [(0.3, 0.6, 0.9)], scale=s)
    ref, sp, off, ids = frame(sc, CAM)
    assert ref["flag"][8, 11] & 1
    var = sp["cov2d"][0]
    a = sp["opacity"][0] * math.exp(-9.0 / (2.0 * var))
    assert abs(a * 255 - 1) < 1e-5
    c = sp["rgb"][0:3]
    same_set(outcomes_at(sp, off, ids, 11, 8), [[0.0, 0.0, 0.0, 1.0], np.append(c * a, 1 - a)])


def test_transmittance_at_the_stop_gives_stop_and_go_on():
    """Three opaque splats (alpha clamped to 0.99): after two, T = 0.01^2 =
    1e-4 up to rounding, the stop threshold. Stopping before the second or
    taking it (and stopping before the third) are both allowed."""
    cs = [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1), (0.1, 0.1, 0.9)]
    sc = stack([0.0, 0.05, 0.1], [logit(0.995)] * 3, cs)
    ref, sp, off, ids = frame(sc, CAM)
    assert ref["flag"][8, 8] & 2
    c1, c2 = sp["rgb"][0:3], sp["rgb"][3:6]
    a = 0.99
    same_set(outcomes_at(sp, off, ids, 8, 8),
             [np.append(c1 * a, 1 - a),
              np.append(c1 * a + c2 * a * (1 - a), (1 - a) * (1 - a))])


def test_centre_on_the_region_boundary_gives_both_colours():
    """A centre projecting exactly onto the selection box's edge: selected or
    not, so the recoloured (t * colour, Sec. 3.3) or the plain colour."""
    t = (0.2, 0.4, 0.8)
    sc = stack([0.0], [logit(0.6)], [(0.7, 0.5, 0.3)])
    edit = sg.Edit(sg.box_region(8.0, 0.0, 12.0, 17.0), sg.tint_matrix(t))
    ref, sp, off, ids = frame(sc, CAM, edit)
    assert sp["sel_flag"][0] == 1 and ref["flag"][8, 8] & 8
    a = sp["opacity"][0]
    plain = frame(sc, CAM)[1]["rgb"][0:3]
    same_set(outcomes_at(sp, off, ids, 8, 8),
             [np.append(plain * a, 1 - a),
              np.append(np.asarray(t, np.float32).astype(np.float64) * plain * a, 1 - a)])


def test_every_pixel_of_a_frame_has_its_render_among_its_outcomes():
    """On the 10k-Gaussian workload: every flagged pixel's outcomes include
    the binned render's value bit for bit, and a pixel without a doubtful
    decision has exactly that one outcome."""
    w = sg.tiny_workload()
    ref, sp, off, ids = frame(w.scene, w.camera, w.edit)
    ys, xs = np.nonzero(ref["flag"] > 0)
    assert 5 < len(ys) < 0.01 * ref["flag"].size
    out, cnt = oracle.pixel_outcomes(sp, off, ids, xs, ys)
    assert cnt.min() >= 1
    can = np.concatenate([ref["rgb"][ys, xs], ref["T"][ys, xs][:, None]], 1)
    d = np.abs(out - can[:, None, :]).max(-1)
    d = np.where(np.arange(out.shape[1])[None, :] < cnt[:, None], d, np.inf)
    assert d.min(1).max() == 0.0
    rng = np.random.default_rng(0)
    uy, ux = np.nonzero(ref["flag"] == 0)
    k = rng.choice(len(uy), 3000, replace=False)
    out, cnt = oracle.pixel_outcomes(sp, off, ids, ux[k], uy[k])
    can = np.concatenate([ref["rgb"][uy[k], ux[k]], ref["T"][uy[k], ux[k]][:, None]], 1)
    one = cnt == 1
    assert one.mean() > 0.99
    assert np.array_equal(out[one, 0], can[one])


def test_depth_keys_round_to_nearest_and_mark_midpoints():
    f = np.float32(3.25)
    up = np.nextafter(f, np.float32(np.inf))
    mid = 0.5 * (float(f) + float(up))
    depths = np.array([float(f), mid, mid + 1e-10 * mid, float(f) + 0.3 * (float(up) - float(f))])
    sp = oracle.SplatResult(depth=depths, margins=oracle.margins(CAM))
    k, amb = oracle.depth_keys(sp)
    assert k[0] == f and not amb[0]
    assert amb[1] and k[1] in (f, up)
    assert k[2] == up and not amb[2]
    assert k[3] == f and not amb[3]
    # a (key, index) sort differs from the (depth, index) order only inside
    # runs of equal keys
    rng = np.random.default_rng(4)
    d = 5.0 + rng.integers(0, 40, 2000) * 2.0 ** -21 + rng.uniform(0, 1e-9, 2000)
    kk = d.astype(np.float32)
    o_depth = np.lexsort((np.arange(2000), d))
    o_key = np.lexsort((np.arange(2000), kk))
    assert not np.array_equal(o_depth, o_key)
    assert np.array_equal(kk[o_depth], kk[o_key])


def test_median_depth_at_tau_gives_both_depths():
    """Two splats of alpha 1/2 at one pixel and tau = 1/2: after the first
    T = 1/2 = tau up to rounding, so the median depth (Sec. 3.2.2) is the
    first splat's or the second's; at tau = 0.6 only the first's."""
    sc = stack([0.0, 0.05], [0.0, 0.0], [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1)])
    ref, sp, off, ids = frame(sc, CAM)
    assert abs(sp["opacity"][0] - 0.5) < 1e-7
    d1, d2 = sp["depth"][0], sp["depth"][1]
    out, cnt = oracle.pixel_outcomes(sp, off, ids, [8], [8], tau=0.5)
    depths = set(np.round(out[0, :cnt[0], 4], 12))
    assert depths == {round(d1, 12), round(d2, 12)}
    out, cnt = oracle.pixel_outcomes(sp, off, ids, [8], [8], tau=0.6)
    assert set(np.round(out[0, :cnt[0], 4], 12)) == {round(d1, 12)}
    # and the colours are those of the plain walk (the depth branch only)
    assert np.allclose(out[0, :cnt[0], :3], ref["rgb"][8, 8])


def test_every_depth_pixel_has_its_render_among_its_outcomes():
    """On the 10k-Gaussian workload with tau = 0.5: every pixel whose depth
    decision is flagged has the binned render's depth among its outcomes'
    depths."""
    w = sg.tiny_workload()
    sp = oracle.preprocess(w.scene, w.camera, w.edit)
    off, ids = oracle.tile_lists(sp, oracle.depth_order(sp), 16, 16)
    ref = oracle.render_tiles(sp, off, ids, tau=0.5)
    ys, xs = np.nonzero(ref["dflag"] > 0)
    assert len(ys) > 3
    out, cnt = oracle.pixel_outcomes(sp, off, ids, xs, ys, tau=0.5)
    assert cnt.min() >= 1
    d = np.abs(out[:, :, 4] - ref["depth"][ys, xs][:, None])
    d = np.where(np.arange(out.shape[1])[None, :] < cnt[:, None], d, np.inf)
    assert d.min(1).max() == 0.0
    # at least one of them has more than one depth
    n_depths = [len(set(out[j, :cnt[j], 4])) for j in range(len(ys))]
    assert max(n_depths) > 1
