"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it cannot agree with by
construction: a library routine (scipy's spherical harmonics), a closed
form, an invariant the paper implies, brute force over all orderings, or a
different algorithm for the same definition. References are to ReCoGS
(arXiv 2511.18441).
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
from paper_2511_18441_b300 import scenegen as sg


# ---------------------------------------------------------------------------
# helpers: hand-built scenes

def make_scene(xyz, log_scale, quat, logit, sh):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    return sg.Scene(f(xyz), f(log_scale), f(quat), f(logit), f(sh))


def single_splat(mu, scale, logit, sh16x3):
    return make_scene(np.array(mu, np.float64).reshape(3, 1),
                      np.full((3, 1), math.log(scale)),
                      np.array([1.0, 0, 0, 0]).reshape(4, 1),
                      np.array([logit]),
                      np.asarray(sh16x3, np.float64).reshape(16, 3, 1))


def all_box(cam):
    return sg.box_region(-1e9, -1e9, 1e9, 1e9)


# ---------------------------------------------------------------------------
# Eq. 2: spherical harmonics

def real_sh_from_scipy(l, m, x, y, z):
    """Real SH built from scipy's complex Y_l^m (Condon-Shortley phase kept):
    m>0: sqrt2 Re Y_l^m, m<0: sqrt2 Im Y_l^|m|, m=0: Y_l^0."""
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x) % (2 * math.pi)
    Yc = complex(sps.sph_harm_y(l, abs(m), theta, phi))
    if m > 0:
        return math.sqrt(2) * Yc.real
    if m < 0:
        return math.sqrt(2) * Yc.imag
    return Yc.real


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y = oracle.sh_basis(*d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(real_sh_from_scipy(l, m, *d), abs=1e-12)


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates polynomials of
    # degree <= 6 on the sphere exactly.
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for j in range(nphi):
            phi = 2 * math.pi * j / nphi
            Y = oracle.sh_basis(s * math.cos(phi), s * math.sin(phi), z)
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_is_direction_only():
    Y1 = oracle.sh_basis(0.3, -0.2, 0.9)
    Y2 = oracle.sh_basis(3.0, -2.0, 9.0)
    np.testing.assert_allclose(Y1, Y2, atol=1e-15)


def test_degree0_colour_is_view_independent():
    rng = np.random.default_rng(5)
    n = 64
    sc = sg.make_scene(n, 11, 0.5, 2, (0.2, 0.4))
    sc.sh[1:] = 0.0
    cams = [sg.look_at_camera(64, 64, 60, (2.5 * math.sin(a), 0.3, -2.5 * math.cos(a)), (0, 0, 0))
            for a in (0.0, 1.0, 2.5)]
    rgbs = [oracle.preprocess(sc, c)["rgb"] for c in cams]
    for r in rgbs[1:]:
        np.testing.assert_allclose(r, rgbs[0], atol=1e-14)
    expect = np.maximum(sc.sh[0].astype(np.float64).T.reshape(-1) / (2 * math.sqrt(math.pi)) + 0.5, 0)
    np.testing.assert_allclose(rgbs[0], expect, atol=1e-14)


# ---------------------------------------------------------------------------
# Eq. 1: rotation and covariance

def hamilton(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_rotation_equals_quaternion_conjugation():
    rng = np.random.default_rng(7)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.1, 10)
        R = oracle.quat_to_rotation(q)
        qn = q / np.linalg.norm(q)
        qc = qn * np.array([1, -1, -1, -1])
        v = rng.normal(size=3)
        rv = hamilton(hamilton(qn, np.r_[0.0, v]), qc)[1:]
        np.testing.assert_allclose(R @ v, rv, atol=1e-12)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)


def test_covariance_eigen_decomposition():
    rng = np.random.default_rng(8)
    for _ in range(20):
        q = rng.normal(size=4)
        ls = rng.normal(-2, 1, size=3)
        S = oracle.covariance3d(q, ls)
        R = oracle.quat_to_rotation(q)
        for k in range(3):  # columns of R are eigenvectors with eigenvalue exp(2 ls_k)
            np.testing.assert_allclose(S @ R[:, k], math.exp(2 * ls[k]) * R[:, k], rtol=1e-12,
                                       atol=1e-15)
        np.testing.assert_allclose(S, S.T, atol=1e-15)


# ---------------------------------------------------------------------------
# projection: closed form and finite differences

def test_single_isotropic_gaussian_closed_form():
    """Pin P4: on-axis isotropic splat of scale s at depth z: Sigma' =
    ((f s / z)^2 + 0.3) I and each pixel shows alpha * rgb with
    alpha = min(0.99, sigma exp(-|d|^2 / (2 v)))."""
    W = H = 64
    cam = sg.axis_camera(W, H, 60.0, 3.0)
    s, logit = 0.02, 0.7
    rng = np.random.default_rng(1)
    sh = rng.normal(0, 0.2, size=(16, 3))
    sc = single_splat((0, 0, 0), s, logit, sh)
    sp = oracle.preprocess(sc, cam)
    f = cam.fy
    v = (f * s / 3.0) ** 2 + 0.3
    # float32 inputs: use the stored values
    s32 = float(np.float32(s))
    s32 = math.exp(float(np.float32(math.log(s))))
    v = (f * s32 / 3.0) ** 2 + 0.3
    np.testing.assert_allclose(sp["cov2d"], [v, 0.0, v], rtol=1e-12, atol=1e-12)
    assert sp["u"][0] == pytest.approx(cam.cx) and sp["v"][0] == pytest.approx(cam.cy)
    # colour at d = +z: only m = 0 terms, Y_l0(z) = sqrt((2l+1)/(4 pi))
    sh32 = sc.sh[:, :, 0].astype(np.float64)
    fcol = sum(sh32[l * l + l] * math.sqrt((2 * l + 1) / (4 * math.pi)) for l in range(4))
    rgb = np.maximum(fcol + 0.5, 0.0)
    np.testing.assert_allclose(sp["rgb"], rgb, atol=1e-13)
    sigma = 1 / (1 + math.exp(-float(np.float32(logit))))
    order = oracle.depth_order(sp)
    py, px = np.mgrid[0:H, 0:W]
    out = oracle.render_pixels(sp, order, px.ravel(), py.ravel())
    d2 = (px.ravel() - cam.cx) ** 2 + (py.ravel() - cam.cy) ** 2
    alpha = np.minimum(0.99, sigma * np.exp(-d2 / (2 * v)))
    keep = alpha >= 1 / 255
    expect = np.where(keep[:, None], alpha[:, None] * rgb[None, :], 0.0)
    np.testing.assert_allclose(out["rgb"], expect, atol=1e-13)
    np.testing.assert_allclose(out["T"], np.where(keep, 1 - alpha, 1.0), atol=1e-13)


def test_two_axis_gaussians_worked_example():
    """The stored closed-form example (tests/golden/two_axis_gaussians_16x16.txt:
    two on-axis Gaussians composited front to back over a background, Eq. 1-3)
    against the binned oracle render of the same scene."""
    from tests import golden_fixtures
    scene, cam, bg, rgb, T = golden_fixtures.two_axis_gaussians()
    img = oracle.render_image(scene, cam, None, bg=bg)[0]
    np.testing.assert_allclose(img["rgb"], rgb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(img["T"], T, rtol=0, atol=1e-12)
    assert not img["flag"].any()


def test_off_axis_covariance_matches_analytic_jacobian():
    """Isotropic splat at view position (x0, 0, z): Sigma' = s^2 J J^T + 0.3 I
    with J = [[f/z, 0, -f x0/z^2], [0, f/z, 0]]."""
    cam = sg.axis_camera(256, 256, 60.0, 4.0)
    for x0 in (-0.8, 0.3, 1.1, 2.9):
        s = 0.05
        sc = single_splat((x0, 0, 0), s, 0.0, np.zeros((16, 3)))
        sp = oracle.preprocess(sc, cam)
        z = 4.0
        f = cam.fx
        lim = 1.3 * cam.width / (2 * f)
        x32 = float(np.float32(x0))
        r = max(-lim, min(lim, x32 / z))
        J = np.array([[f / z, 0, -f * r / z], [0, f / z, 0]])
        s32 = math.exp(float(np.float32(math.log(s))))
        S2 = s32 ** 2 * J @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(sp["cov2d"], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-12)
        assert sp["u"][0] == pytest.approx(f * x32 / z + cam.cx, abs=1e-9)


def test_projected_covariance_matches_finite_difference_jacobian():
    """For a rotated camera and anisotropic splat inside the clamp range,
    Sigma' - 0.3 I equals D Sigma D^T with D the finite-difference Jacobian of
    the world -> pixel map at the centre."""
    cam = sg.look_at_camera(320, 240, 50.0, (1.5, -0.7, -3.0), (0.1, 0.2, 0.0))
    rng = np.random.default_rng(4)
    Wv = np.asarray(cam.world_to_view, np.float64)

    def pix(p):
        t = Wv[:, :3] @ p + Wv[:, 3]
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])

    for _ in range(10):
        mu = rng.uniform(-0.3, 0.3, size=3).astype(np.float32).astype(np.float64)
        q = rng.normal(size=4)
        ls = rng.normal(-3, 0.5, size=3)
        sc = make_scene(mu.reshape(3, 1), ls.reshape(3, 1), q.reshape(4, 1), [0.0],
                        np.zeros((16, 3, 1)))
        sp = oracle.preprocess(sc, cam)
        h = 1e-6
        D = np.stack([(pix(mu + h * e) - pix(mu - h * e)) / (2 * h) for e in np.eye(3)], 1)
        Sig = oracle.covariance3d(sc.quat[:, 0].astype(np.float64), sc.log_scale[:, 0].astype(np.float64))
        S2 = D @ Sig @ D.T
        got = np.array(sp["cov2d"]) - np.array([0.3, 0.0, 0.3])
        np.testing.assert_allclose(got, [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6,
                                   atol=1e-9 * abs(S2).max())


def test_near_plane_and_behind_camera_contribute_nothing():
    cam = sg.axis_camera(64, 64, 60.0, 1.0)
    sh = np.zeros((16, 3))
    sh[0] = 3.0
    for z in (-0.85, -1.5):  # view depth 0.15 < 0.2 and -0.5
        sc = single_splat((0, 0, z), 0.05, 3.0, sh)
        sp = oracle.preprocess(sc, cam)
        assert sp["valid"][0] == 0 and sp["visible"][0] == 0
        out = oracle.render_pixels(sp, oracle.depth_order(sp), [32], [32])
        assert out["rgb"].max() == 0.0 and out["T"][0] == 1.0


# ---------------------------------------------------------------------------
# Eq. 3: blending

def brute_force_pixel(sp, px, py, bg):
    """O(N^2) form of Eq. 3: a splat contributes f_i alpha_i prod_{j in front}
    (1 - alpha_j), the product over contributing splats j that precede i in
    (depth, index) order found by comparing every pair; a splat is dropped if
    alpha < 1/255, and every splat from the first one whose inclusion would take
    the product below 1e-4 onwards is dropped."""
    n = sp["n"]
    idx = [i for i in range(n) if sp["valid"][i]]
    alpha = {}
    for i in idx:
        dx, dy = px - sp["u"][i], py - sp["v"][i]
        A, B, Cc = sp["conic"][3 * i:3 * i + 3]
        p = min(0.0, -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
        alpha[i] = min(0.99, sp["opacity"][i] * math.exp(p))
    cand = [i for i in idx if alpha[i] >= 1 / 255]

    def before(j, i):
        return (sp["depth"][j], j) < (sp["depth"][i], i)

    prod_incl = {}
    for i in cand:  # product including i itself over all candidates up to i
        pr = 1.0 - alpha[i]
        for j in cand:
            if before(j, i):
                pr *= 1.0 - alpha[j]
        prod_incl[i] = pr
    # the transmittance is monotone, so the stop rule keeps exactly the
    # candidates whose inclusive product stays >= 1e-4
    kept = [i for i in cand if prod_incl[i] >= 1e-4]
    col = np.zeros(3)
    for i in kept:
        Ti = prod_incl[i] / (1.0 - alpha[i])
        col += sp["rgb"][3 * i:3 * i + 3] * alpha[i] * Ti
    Tf = min([prod_incl[i] for i in kept], default=1.0)
    return col + Tf * np.asarray(bg), Tf


@pytest.mark.parametrize("seed,log_scale", [(0, -2.8), (1, -2.8), (2, -1.5), (3, -1.2)])
def test_blend_matches_brute_force_on_tiny_scenes(seed, log_scale):
    """Pin P5: random scenes of 48 splats, including exactly equal depths;
    the larger scales overlap enough for blending to terminate."""
    rng = np.random.default_rng(100 + seed)
    n = 48
    xyz = rng.uniform(-0.25, 0.25, size=(3, n))
    xyz[2, :6] = xyz[2, 6:12]  # exact depth ties
    sc = make_scene(xyz, rng.normal(log_scale, 0.4, size=(3, n)), rng.normal(size=(4, n)),
                    rng.normal(1.0, 2.0, size=n), rng.normal(0, 0.3, size=(16, 3, n)))
    cam = sg.axis_camera(32, 32, 60.0, 2.0)
    sp = oracle.preprocess(sc, cam)
    order = oracle.depth_order(sp)
    bg = (0.1, 0.2, 0.3)
    pxs = rng.integers(0, 32, size=40)
    pys = rng.integers(0, 32, size=40)
    out = oracle.render_pixels(sp, order, pxs, pys, bg=bg)
    if log_scale > -1.3:
        assert (out["T"] < 1e-3).any()  # some pixels reach the stop rule
    for k in range(len(pxs)):
        col, Tf = brute_force_pixel(sp, float(pxs[k]), float(pys[k]), bg)
        np.testing.assert_allclose(out["rgb"][k], col, atol=1e-12)
        assert out["T"][k] == pytest.approx(Tf, abs=1e-12)


def test_termination_stops_before_the_splat():
    """Stack of wide splats with alpha ~ 0.85 at one pixel: T goes 1, .15,
    .0225, 3.4e-3, 5.1e-4; the fifth would take it to 7.7e-5 < 1e-4, so
    exactly four contribute and the output is their closed-form sum."""
    cam = sg.axis_camera(16, 16, 60.0, 2.0)
    n = 6
    logit = math.log(0.85 / 0.15)
    sh = np.zeros((16, 3, n))
    sh[0] = ((np.arange(n) + 1) / 10.0 - 0.5) * 2 * math.sqrt(math.pi)  # rgb = (k+1)/10
    sc = make_scene(np.stack([np.zeros(n), np.zeros(n), np.linspace(0, 0.5, n)]),
                    np.full((3, n), math.log(3.0)), np.tile([[1.0], [0], [0], [0]], n),
                    np.full(n, logit), sh)
    sp = oracle.preprocess(sc, cam)
    out = oracle.render_pixels(sp, oracle.depth_order(sp), [8], [8])
    T = 1.0
    col = np.zeros(3)
    for k in range(n):
        A, B, Cc = sp["conic"][3 * k:3 * k + 3]
        dx, dy = 8 - sp["u"][k], 8 - sp["v"][k]
        a = min(0.99, sp["opacity"][k] * math.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy))
        assert 0.84 < a < 0.85
        if T * (1 - a) < 1e-4:
            assert k == 4 and T * (1 - a) > 1e-5
            break
        col += sp["rgb"][3 * k:3 * k + 3] * a * T
        T *= 1 - a
    assert out["ncontrib"][0] == 4
    np.testing.assert_allclose(out["rgb"][0], col, atol=1e-12)
    assert out["T"][0] == pytest.approx(T, rel=1e-12)


def test_transparent_splat_changes_no_pixel():
    """Pin P3: a splat with opacity sigmoid(-30) < 1/255 leaves every bit."""
    w = sg.tiny_workload(n=2000)
    extra = single_splat((0.0, 0.0, 0.0), 0.2, -30.0, np.full((16, 3), 0.5))
    sc2 = w.scene.concat(extra)
    a, *_ = oracle.render_image(w.scene, w.camera, w.edit)
    b, *_ = oracle.render_image(sc2, w.camera, w.edit)
    assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["T"], b["T"])
    py, px = np.mgrid[0:256:7, 0:256:7]
    spa = oracle.preprocess(w.scene, w.camera, w.edit)
    spb = oracle.preprocess(sc2, w.camera, w.edit)
    ra = oracle.render_pixels(spa, oracle.depth_order(spa), px.ravel(), py.ravel())
    rb = oracle.render_pixels(spb, oracle.depth_order(spb), px.ravel(), py.ravel())
    assert np.array_equal(ra["rgb"], rb["rgb"])


def test_definitional_and_binned_agree():
    """Pin P8 on the 10k-splat workload: the per-pixel walk over every splat
    and the per-tile lists give the same image."""
    w = sg.tiny_workload()
    img, sp, order, off, ids = oracle.render_image(w.scene, w.camera, w.edit)
    H, W = 256, 256
    py, px = np.mgrid[0:H, 0:W]
    r = oracle.render_pixels(sp, order, px.ravel(), py.ravel())
    np.testing.assert_allclose(r["rgb"].reshape(H, W, 3), img["rgb"], atol=1e-12)
    np.testing.assert_allclose(r["T"].reshape(H, W), img["T"], atol=1e-12)
    assert (r["ncontrib"].reshape(H, W) == img["ncontrib"]).all()


def test_tile_lists_are_complete_and_sorted():
    """Every splat that reaches alpha >= 1/255 at some pixel of a tile is in
    that tile's list, and lists are in (depth, index) order."""
    w = sg.tiny_workload(n=3000)
    cam = w.camera
    sp = oracle.preprocess(w.scene, cam, w.edit)
    order = oracle.depth_order(sp)
    tx, ty = 16, 16
    off, ids = oracle.tile_lists(sp, order, tx, ty)
    for t in range(tx * ty):
        lst = ids[off[t]:off[t + 1]]
        keys = [(sp["depth"][i], i) for i in lst]
        assert keys == sorted(keys)
    rng = np.random.default_rng(0)
    for i in rng.choice(np.flatnonzero(sp["valid"]), 300, replace=False):
        u, v = sp["u"][i], sp["v"][i]
        A, B, Cc = sp["conic"][3 * i:3 * i + 3]
        x0, x1 = int(max(0, math.floor(u - 20))), int(min(255, math.ceil(u + 20)))
        y0, y1 = int(max(0, math.floor(v - 20))), int(min(255, math.ceil(v + 20)))
        yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        dx, dy = xx - u, yy - v
        p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
        hit = sp["opacity"][i] * np.exp(np.minimum(p, 0)) >= 1 / 255
        for y, x in zip(yy[hit], xx[hit]):
            t = (y // 16) * tx + x // 16
            assert i in set(ids[off[t]:off[t + 1]].tolist())


# ---------------------------------------------------------------------------
# tint (Sec. 3.3) and the identity cases

def test_unselected_sh_unchanged_and_identity_tint():
    """Pin P2."""
    w = sg.tiny_workload(n=500)
    sel = (np.arange(500) % 3 == 0).astype(np.uint8)
    out = oracle.recolor(w.scene.sh, sel, w.edit.color_matrix)
    same = out[:, :, sel == 0]
    assert np.array_equal(same, w.scene.sh[:, :, sel == 0].astype(np.float64))
    ident = oracle.recolor(w.scene.sh, np.ones(500, np.uint8), np.eye(3))
    assert np.array_equal(ident, w.scene.sh.astype(np.float64))
    e1 = sg.Edit(w.edit.region, np.eye(3, dtype=np.float32))
    a, *_ = oracle.render_image(w.scene, w.camera, None)
    b, *_ = oracle.render_image(w.scene, w.camera, e1)
    assert np.array_equal(a["rgb"], b["rgb"])


def test_recoloured_colour_is_matrix_times_colour():
    """Before the clamp the recoloured colour is M (f + 0.5) from every view
    direction, for a general (hue) matrix."""
    rng = np.random.default_rng(9)
    n = 200
    sh = rng.normal(0, 0.3, size=(16, 3, n)).astype(np.float32)
    M = sg.hue_rotation_matrix(70.0).astype(np.float64)
    out = oracle.recolor(sh, np.ones(n, np.uint8), M)
    for _ in range(5):
        d = rng.normal(size=3)
        Y = oracle.sh_basis(*d)
        f = np.einsum("k,kcn->cn", Y, sh.astype(np.float64))
        f2 = np.einsum("k,kcn->cn", Y, out)
        np.testing.assert_allclose(f2 + 0.5, M @ (f + 0.5), atol=1e-12)


def test_tint_invariant_whole_image():
    """Pin P1: with every splat selected, a tint t >= 0 and a black
    background, the recoloured render is t times the render, and the sort order
    and tile lists do not change (geometry frozen, Sec. 3.3)."""
    w = sg.tiny_workload(n=4000)
    t = np.array([0.9, 0.4, 0.2])
    e = sg.Edit(all_box(w.camera), sg.tint_matrix(t))
    a, spa, oa, offa, ida = oracle.render_image(w.scene, w.camera, None)
    b, spb, ob, offb, idb = oracle.render_image(w.scene, w.camera, e)
    assert spb["selected"].all()
    np.testing.assert_allclose(b["rgb"], a["rgb"] * t.astype(np.float32).astype(np.float64),
                               atol=1e-12)
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(oa, ob) and np.array_equal(offa, offb) and np.array_equal(ida, idb)


# ---------------------------------------------------------------------------
# selection

def winding_number(u, v, poly):
    """Sum of signed angles subtended by the edges (a different algorithm from
    the oracle's crossing count)."""
    ang = 0.0
    k = len(poly)
    for i in range(k):
        ax, ay = poly[i][0] - u, poly[i][1] - v
        bx, by = poly[(i + 1) % k][0] - u, poly[(i + 1) % k][1] - v
        ang += math.atan2(ax * by - ay * bx, ax * bx + ay * by)
    return round(ang / (2 * math.pi))


def test_polygon_selection_against_winding_number():
    """Pin P7: selection of splat centres by the oracle equals the winding
    number test for the simple star polygon, away from flagged centres."""
    w = sg.paper_scale_workload(n=20000)
    sel, flag = oracle.select(w.scene, w.edit, w.camera)
    Wv = np.asarray(w.camera.world_to_view, np.float64)
    t = Wv[:, :3] @ w.scene.xyz.astype(np.float64) + Wv[:, 3:4]
    u = w.camera.fx * t[0] / t[2] + w.camera.cx
    v = w.camera.fy * t[1] / t[2] + w.camera.cy
    poly = w.edit.region.xy.astype(np.float64)
    idx = np.random.default_rng(0).choice(w.scene.n, 3000, replace=False)
    for i in idx:
        if flag[i]:
            continue
        expect = (t[2, i] > 0) and winding_number(u[i], v[i], poly) != 0
        assert bool(sel[i]) == expect
    assert 0.05 < sel.mean() < 0.8


def test_polygon_area_by_grid_count():
    """The even-odd region's area on a fine pixel grid equals the shoelace
    area of the generated polygon (15% of the image)."""
    cam = sg.axis_camera(192, 108, 60.0, 5.0)
    reg = sg.polygon_region(192, 108, 12, 0.15, 1)
    assert sg.shoelace_area(reg.xy) == pytest.approx(0.15 * 192 * 108, rel=1e-5)
    # points on a grid 4x finer than pixels, placed at depth 1 in front of a
    # camera at the origin so that they project to the grid positions
    g = 4
    ys, xs = np.mgrid[0:108 * g, 0:192 * g]
    uu = (xs + 0.5) / g - 0.5
    vv = (ys + 0.5) / g - 0.5
    cam0 = sg.Camera(192, 108, cam.fx, cam.fy, cam.cx, cam.cy,
                     np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32),
                     np.zeros(3, np.float32))
    pts = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)]).reshape(3, -1)
    sc = make_scene(pts, np.zeros_like(pts), np.tile([[1.0], [0], [0], [0]], pts.shape[1]),
                    np.zeros(pts.shape[1]), np.zeros((16, 3, pts.shape[1])))
    sel, _ = oracle.select(sc, sg.Edit(reg, np.eye(3, dtype=np.float32)), cam0)
    area = sel.sum() / (g * g)
    assert area == pytest.approx(0.15 * 192 * 108, rel=0.01)


def test_box_selection_half_open_pixel_box():
    """The 64x64 pixel box [96, 160)^2 selects centres whose nearest pixel
    lies in it: continuous [95.5, 159.5)."""
    cam = sg.axis_camera(256, 256, 60.0, 2.5)
    reg = sg.pixel_box_region(96, 96, 64, 64)
    us = np.array([95.4, 95.6, 159.4, 159.6, 127.0])
    vs = np.array([127.0, 127.0, 127.0, 127.0, 159.45])
    z = 2.5
    pts = np.stack([(us - cam.cx) / cam.fx * z, (vs - cam.cy) / cam.fy * z, np.zeros_like(us)])
    sc = make_scene(pts, np.zeros((3, 5)), np.tile([[1.0], [0], [0], [0]], 5), np.zeros(5),
                    np.zeros((16, 3, 5)))
    sel, flag = oracle.select(sc, sg.Edit(reg, np.eye(3, dtype=np.float32)), cam)
    assert sel.tolist() == [0, 1, 1, 0, 1]
    assert not flag.any()


# ---------------------------------------------------------------------------
# per-splat quantities against independent restatements

def test_splat_colour_matches_scipy_sh_at_view_direction():
    """rgb = max(sum_lm C_lm Y_lm(d) + 0.5, 0) with d from the camera centre to
    the splat, Y from scipy, channels and coefficient indices as laid out."""
    w = sg.tiny_workload(n=40)
    cam = sg.look_at_camera(64, 64, 60, (1.0, -0.5, -2.5), (0, 0, 0))
    sp = oracle.preprocess(w.scene, cam)
    for i in range(w.scene.n):
        d = w.scene.xyz[:, i].astype(np.float64) - cam.cam_pos.astype(np.float64)
        d /= np.linalg.norm(d)
        for c in range(3):
            f = sum(float(w.scene.sh[l * l + l + m, c, i]) * real_sh_from_scipy(l, m, *d)
                    for l in range(4) for m in range(-l, l + 1))
            assert sp["rgb"][3 * i + c] == pytest.approx(max(f + 0.5, 0.0), abs=1e-12)


def test_conic_is_inverse_covariance():
    w = sg.tiny_workload(n=200)
    sp = oracle.preprocess(w.scene, w.camera)
    for i in np.flatnonzero(sp["valid"])[:200]:
        a, b, c = sp["cov2d"][3 * i:3 * i + 3]
        A, B, Cc = sp["conic"][3 * i:3 * i + 3]
        np.testing.assert_allclose(np.array([[A, B], [B, Cc]]) @ np.array([[a, b], [b, c]]),
                                   np.eye(2), atol=1e-12)


def test_jacobian_clamp_outside_field_of_view():
    """A splat beyond 1.3x the half field of view uses the clamped x/z in J."""
    cam = sg.axis_camera(256, 256, 60.0, 4.0)
    x0, s = 3.9, 0.05
    sc = single_splat((x0, 0, 0), s, 0.0, np.zeros((16, 3)))
    sp = oracle.preprocess(sc, cam)
    f, z = cam.fx, 4.0
    lim = 1.3 * cam.width / (2 * f)
    assert float(np.float32(x0)) / z > lim
    J = np.array([[f / z, 0, -f * lim / z], [0, f / z, 0]])
    s32 = math.exp(float(np.float32(math.log(s))))
    S2 = s32 ** 2 * J @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(sp["cov2d"], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-12)


def test_extent_touches_the_cutoff_ellipse():
    """The x-extremal point of {d : sigma exp(-d^T conic d / 2) >= 1/255} is
    d* = sqrt(k/a) (a, b) with k = 2 ln(255 sigma); its x offset is the
    extent, and alpha there is exactly 1/255."""
    w = sg.tiny_workload(n=300)
    sp = oracle.preprocess(w.scene, w.camera)
    for i in np.flatnonzero(sp["visible"])[:200]:
        a, b, c = sp["cov2d"][3 * i:3 * i + 3]
        A, B, Cc = sp["conic"][3 * i:3 * i + 3]
        k = 2 * math.log(255 * sp["opacity"][i])
        d = math.sqrt(k / a) * np.array([a, b])
        assert d[0] == pytest.approx(sp["extent"][2 * i], rel=1e-12)
        p = -0.5 * (A * d[0] ** 2 + Cc * d[1] ** 2) - B * d[0] * d[1]
        assert sp["opacity"][i] * math.exp(p) == pytest.approx(1 / 255, rel=1e-10)
        e = math.sqrt(k / c) * np.array([b, c])
        assert e[1] == pytest.approx(sp["extent"][2 * i + 1], rel=1e-12)


def test_tile_range_is_the_tiles_with_a_pixel_centre_in_the_box():
    """Brute force over pixel centres: tile t is in [tx0, tx1] iff some
    centre x in 16t..16t+15 (inside the image) has |x - u| <= extent."""
    w = sg.tiny_workload(n=2000)
    sp = oracle.preprocess(w.scene, w.camera)
    W = w.camera.width
    tiles = (W + 15) // 16
    for i in np.flatnonzero(sp["visible"])[:500]:
        u, ex = sp["u"][i], sp["extent"][2 * i]
        hit = [t for t in range(tiles)
               if any(abs(x - u) <= ex for x in range(16 * t, min(16 * t + 16, W)))]
        tx0, tx1 = sp["rect"][4 * i], sp["rect"][4 * i + 1]
        # the continuous rule may add a tile whose span meets the box between
        # two centres only when the box is narrower than one pixel
        if hit:
            assert tx0 <= hit[0] and tx1 >= hit[-1]
            assert tx1 - tx0 + 1 - len(hit) <= (1 if 2 * ex < 1 else 0)


# ---------------------------------------------------------------------------
# median depth (Sec. 3.2.2) and the SH-only refit (Sec. 3.3, Eq. 6-7)

def stack_scene(opacities, depths, scale=3.0):
    """Wide on-axis splats (near-constant alpha over a 16x16 view) at the
    given world depths, rgb = 0.5 everywhere."""
    n = len(opacities)
    logit = [math.log(o / (1 - o)) for o in opacities]
    return make_scene(np.stack([np.zeros(n), np.zeros(n), np.asarray(depths, np.float64)]),
                      np.full((3, n), math.log(scale)), np.tile([[1.0], [0], [0], [0]], n),
                      np.asarray(logit), np.zeros((16, 3, n)))


@pytest.mark.parametrize("tau,expect", [(0.5, 1), (0.2, 2), (0.01, None)])
def test_median_depth_is_the_splat_that_takes_T_below_tau(tau, expect):
    """Opacities 0.3, 0.5, 0.9 front to back: T after each is about 0.7,
    0.35, 0.035, so tau = 0.5 picks the second splat, tau = 0.2 the third,
    and tau = 0.01 none (depth 0). The depth is the splat's view depth,
    here the camera distance plus its world z."""
    cam = sg.axis_camera(16, 16, 60.0, 2.0)
    z = [0.0, 0.25, 0.5]
    sc = stack_scene([0.3, 0.5, 0.9], z)
    sp = oracle.preprocess(sc, cam)
    order = oracle.depth_order(sp)
    off, ids = oracle.tile_lists(sp, order, 1, 1)
    out = oracle.render_tiles(sp, off, ids, tau=tau)
    plain = oracle.render_tiles(sp, off, ids)
    np.testing.assert_array_equal(out["rgb"], plain["rgb"])
    d = out["depth"][8, 8]
    if expect is None:
        assert d == 0.0
    else:
        assert d == pytest.approx(2.0 + z[expect], abs=1e-12)
        # and it is the first splat after which T < tau at that pixel
        T = 1.0
        for k in range(3):
            A, B, Cc = sp["conic"][3 * k:3 * k + 3]
            dx, dy = 8 - sp["u"][k], 8 - sp["v"][k]
            a = min(0.99, sp["opacity"][k] * math.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy))
            if T >= tau > T * (1 - a):
                assert k == expect
                break
            T *= 1 - a
    assert not out["dflag"].any()


def refit_scene():
    w = sg.tiny_workload(n=400, width=48, height=40)
    return w.scene, w.camera


def l1_of(sp, off, ids, target):
    img = oracle.render_tiles(sp, off, ids)["rgb"]
    return oracle.l1_loss_grad(img, target)[0]


def test_colour_gradient_matches_finite_differences():
    """Eq. 3 is linear in the splat colours, so with the signs of y - target
    held fixed the L1 loss is linear in each colour and a central difference
    gives the gradient up to rounding."""
    scene, cam = refit_scene()
    sp = oracle.preprocess(scene, cam)
    order = oracle.depth_order(sp)
    off, ids = oracle.tile_lists(sp, order, 3, 3)
    y = oracle.render_tiles(sp, off, ids)["rgb"]
    rng = np.random.default_rng(0)
    target = y + rng.choice([-1.0, 1.0], size=y.shape) * rng.uniform(0.05, 0.2, size=y.shape)
    _, g = oracle.l1_loss_grad(y, target)
    grad = oracle.color_grad(sp, off, ids, g)
    contributing = np.nonzero(np.abs(grad).sum(1) > 1e-6)[0]
    assert len(contributing) > 20
    h = 1e-4
    for i in rng.choice(contributing, 12, replace=False):
        for ch in range(3):
            base = sp["rgb"][3 * i + ch]
            sp["rgb"][3 * i + ch] = base + h
            lp = l1_of(sp, off, ids, target)
            sp["rgb"][3 * i + ch] = base - h
            lm = l1_of(sp, off, ids, target)
            sp["rgb"][3 * i + ch] = base
            assert grad[i, ch] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-12)


def test_sh_gradient_matches_finite_differences_through_the_whole_render():
    """dL/dC of Eq. 2 chained with the colour gradient, against a central
    difference of the full pipeline (preprocess + render) in one float32
    SH coefficient; the colour is affine in C away from the clamp."""
    scene, cam = refit_scene()
    sp = oracle.preprocess(scene, cam)
    order = oracle.depth_order(sp)
    off, ids = oracle.tile_lists(sp, order, 3, 3)
    y = oracle.render_tiles(sp, off, ids)["rgb"]
    rng = np.random.default_rng(1)
    target = y + rng.choice([-1.0, 1.0], size=y.shape) * rng.uniform(0.05, 0.2, size=y.shape)
    _, g = oracle.l1_loss_grad(y, target)
    gsh = oracle.sh_grad(scene, sp, oracle.color_grad(sp, off, ids, g))
    cand = np.nonzero(np.abs(gsh[0]).sum(0) > 1e-6)[0]
    assert len(cand) > 10

    def loss(sh):
        s2 = sg.Scene(scene.xyz, scene.log_scale, scene.quat, scene.opacity_logit, sh)
        p2 = oracle.preprocess(s2, cam)
        return l1_of(p2, off, ids, target)

    for i in rng.choice(cand, 6, replace=False):
        for k, ch in ((0, 0), (3, 1), (8, 2), (15, 0)):
            shp = scene.sh.copy()
            shm = scene.sh.copy()
            shp[k, ch, i] = np.float32(shp[k, ch, i] + np.float32(2.0 ** -10))
            shm[k, ch, i] = np.float32(shm[k, ch, i] - np.float32(2.0 ** -10))
            dC = float(shp[k, ch, i]) - float(shm[k, ch, i])
            fd = (loss(shp) - loss(shm)) / dC
            assert gsh[k, ch, i] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_adam_first_step_moves_each_coefficient_by_lr_against_its_sign():
    """From m = v = 0 the bias-corrected first Adam step is lr g / (|g| + eps):
    lr sign(g) for |g| >> eps, and a zero gradient moves nothing."""
    rng = np.random.default_rng(2)
    C0 = rng.normal(size=(16, 3, 5))
    g = rng.normal(size=C0.shape)
    g[:, :, 0] = 0.0
    C1, m, v = oracle.adam_step(C0, g, np.zeros_like(C0), np.zeros_like(C0), 1, 0.01)
    np.testing.assert_allclose(C1, C0 - 0.01 * np.sign(g), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(C1[:, :, 0], C0[:, :, 0])
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_refit_fixed_point_has_zero_loss_and_gradient():
    """The target rendered from the scene itself is the refit's fixed point:
    L1 = 0, sign(0) = 0, so every SH gradient and Adam update is zero."""
    scene, cam = refit_scene()
    sp = oracle.preprocess(scene, cam)
    off, ids = oracle.tile_lists(sp, oracle.depth_order(sp), 3, 3)
    y = oracle.render_tiles(sp, off, ids)["rgb"]
    loss, g = oracle.l1_loss_grad(y, y)
    assert loss == 0.0 and not g.any()
    gsh = oracle.sh_grad(scene, sp, oracle.color_grad(sp, off, ids, g))
    assert not gsh.any()
