"""Pins of the learned-selection oracle (oracle/mlp.py) against facts fixed
outside it: finite differences of its own loss (FP64 path), torch's bfloat16
conversion, closed forms of GELU, the radial frame and the rendered coverage
of a single Gaussian, and the plain selection. ReCoGS (arXiv 2511.18441) names the leak of
its selection as a limitation (Sec. 6); the learned variant is the
the benchmark spec's extension."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2511_18441_b300 import scenegen as sg

torch = pytest.importorskip("torch")


def test_gradient_matches_finite_differences_fp64():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (7, mlp.K))
    X[:, mlp.N_IN:] = 0
    sel = rng.integers(0, 2, 7)
    cov = rng.uniform(0, 1, 7)
    loss, g = mlp.loss_grad(theta, X, sel, cov, rnd=False)
    h = 1e-6
    # a few coordinates of every parameter block
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    coords = np.concatenate([rng.integers(a, b, 8) for a, b in zip(starts[:-1], starts[1:])])
    for j in coords:
        tp = theta.copy()
        tm = theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (mlp.loss_grad(tp, X, sel, cov, rnd=False)[0] -
              mlp.loss_grad(tm, X, sel, cov, rnd=False)[0]) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 10, 5000), [1 + 2 ** -8, 1 + 3 * 2 ** -8, -0.0, 3e-39]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32), ref.astype(np.float64))
    assert mlp.bf16(np.array([1 + 2 ** -8]))[0] == 1.0          # tie to even
    assert mlp.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    assert mlp.gelu(np.array([-10.0]))[0] == pytest.approx(0.0, abs=1e-20)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-10)
    # GELU(1) = Phi(1) with Phi the standard normal CDF
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-14)


def test_radial_frame_maps_the_polygon_onto_the_unit_disc():
    ang = np.linspace(0, 2 * math.pi, 9)[:-1] + 0.1
    rad = np.array([1.0, 1.3, 0.8, 1.1, 0.9, 1.2, 1.0, 0.7]) * 50
    xy = np.stack([100 + rad * np.cos(ang), 80 + rad * np.sin(ang)], 1)
    c = xy.mean(0)
    # vertices and edge midpoints lie on the boundary: radius 1
    mids = 0.5 * (xy + np.roll(xy, 1, 0))
    for P in (xy, mids):
        un, vn, rho = mlp.radial_frame(P[:, 0], P[:, 1], xy)
        np.testing.assert_allclose(np.hypot(un, vn), 1.0, rtol=1e-12)
        np.testing.assert_allclose(rho, np.hypot(*(P - c).T), rtol=1e-12)
    # halfway to the boundary: radius 1/2; the centroid: 0
    un, vn, _ = mlp.radial_frame(0.5 * (mids[:, 0] + c[0]), 0.5 * (mids[:, 1] + c[1]), xy)
    np.testing.assert_allclose(np.hypot(un, vn), 0.5, rtol=1e-12)
    un, vn, _ = mlp.radial_frame(np.array([c[0]]), np.array([c[1]]), xy)
    assert un[0] == 0.0 and vn[0] == 0.0
    # scaling the polygon about its centroid by s scales the frame by 1/s
    p = np.array([c[0] + 13.0]), np.array([c[1] - 7.0])
    a = np.hypot(*mlp.radial_frame(*p, xy)[:2])
    b = np.hypot(*mlp.radial_frame(*p, c + 2.0 * (xy - c))[:2])
    assert b[0] == pytest.approx(a[0] / 2.0, rel=1e-12)


def small_scene(n=300, seed=3):
    w = sg.tiny_workload(n=n, seed=seed, width=64, height=64)
    return w.scene, w.camera


def test_features_layout_and_plain_label():
    scene, cam = small_scene()
    xy = sg.polygon_region(64, 64, 12, 0.2, 5).xy
    F, valid, sel, cov = mlp.features_and_labels(scene, cam, xy)
    n = scene.n
    np.testing.assert_allclose(F[:, 9], scene.log_scale.astype(np.float64).mean(0), rtol=1e-12)
    np.testing.assert_array_equal(F[:, 10], scene.opacity_logit.astype(np.float64))
    np.testing.assert_allclose(F[:, 6] ** 2 + F[:, 7] ** 2, 1.0, rtol=1e-9)
    assert (F[:, 3] >= F[:, 4]).all() and (F[:, 5] <= F[:, 3] + 1e-12).all()
    assert (F[:, 5] >= F[:, 4] - 1e-12).all()
    np.testing.assert_array_equal(F[:, 11:59], scene.sh.reshape(48, n).T.astype(np.float64))
    assert not F[:, 59:].any()
    edit = sg.Edit(sg.Region("polygon", xy), np.eye(3, dtype=np.float32), cam)
    ref, _ = oracle.select(scene, edit, cam)
    np.testing.assert_array_equal(sel, ref)
    assert valid.all() and 0.05 < sel.mean() < 0.95
    assert ((cov >= 0) & (cov <= 1)).all()
    # centre inside the polygon frame <=> plain selection, for a star-shaped polygon
    r = np.hypot(F[:, 0], F[:, 1])
    far = np.abs(r - 1) > 1e-9
    np.testing.assert_array_equal((r < 1)[far], sel.astype(bool)[far])


def test_selection_view_shape_features_closed_form():
    """An isotropic splat at (x0, 0, 0) in front of the axis camera and a
    square of half-width h centred on the image: along +x, rho = h,
    Sigma'_xx = (f s / z)^2 (1 + (x0 / z)^2) + 0.3 (the Jacobian's x row),
    Sigma'_yy = (f s / z)^2 + 0.3, no cross term; the major axis lies along
    the radial direction."""
    cam = sg.axis_camera(201, 201, 60.0, 3.0)
    s, x0, h = 0.15, 0.4, 60.0
    sc = sg.Scene(np.array([[x0], [0.0], [0.0]], np.float32), np.full((3, 1), math.log(s), np.float32),
                  np.array([[1.0], [0], [0], [0]], np.float32), np.zeros(1, np.float32),
                  np.zeros((16, 3, 1), np.float32))
    c = np.array([cam.cx, cam.cy])
    sq = c + np.array([[-h, -h], [h, -h], [h, h], [-h, h]])
    F = mlp.features_and_labels(sc, cam, sq)[0][0]
    z = 3.0
    s32 = math.exp(float(np.float32(math.log(s))))
    x32 = float(np.float32(x0))
    fx = float(np.float32(cam.fx))
    sxx = (fx * s32 / z) ** 2 * (1 + (x32 / z) ** 2) + 0.3
    syy = (float(np.float32(cam.fy)) * s32 / z) ** 2 + 0.3
    u = fx * x32 / z + float(np.float32(cam.cx))
    d = u - c[0]
    assert F[0] == pytest.approx(d / h, rel=1e-9) and F[1] == pytest.approx(0.0, abs=1e-12)
    assert F[3] == pytest.approx(0.5 * math.log(sxx) - math.log(h), rel=1e-9)
    assert F[4] == pytest.approx(0.5 * math.log(syy) - math.log(h), rel=1e-9)
    assert F[5] == pytest.approx(F[3], rel=1e-12)
    assert F[6] == pytest.approx(1.0, abs=1e-12) and F[7] == pytest.approx(0.0, abs=1e-12)
    assert F[8] == pytest.approx((h - d) / math.sqrt(sxx), rel=1e-8)
    assert F[2] == pytest.approx(math.log(z * h / fx), rel=1e-9)
    # far from the boundary the distance feature saturates at 8
    sq_big = c + np.array([[-h, -h], [h, -h], [h, h], [-h, h]]) * 3
    assert mlp.features_and_labels(sc, cam, sq_big)[0][0, 8] == 8.0


def test_rendered_coverage_of_a_single_gaussian_in_closed_form():
    """One isotropic Gaussian on the axis: T = 1 at every pixel, so the
    tint-weight label of a half-plane region is the sum of alpha^2 over the
    pixels inside it over the sum over all pixels, alpha = min(0.99,
    sigma exp(-d^2 / (2 v))) with v = (f s / z)^2 + 0.3 (the single-Gaussian
    pin of the render), counting only alpha >= 1/255."""
    W = H = 41
    cam = sg.axis_camera(W, H, 60.0, 3.0)
    s, logit = 0.03, 1.2
    sc = sg.Scene(np.zeros((3, 1), np.float32), np.full((3, 1), math.log(s), np.float32),
                  np.array([[1.0], [0], [0], [0]], np.float32), np.array([logit], np.float32),
                  np.zeros((16, 3, 1), np.float32))
    s32 = math.exp(float(np.float32(math.log(s))))
    v = (cam.fy * s32 / 3.0) ** 2 + 0.3
    sigma = 1 / (1 + math.exp(-float(np.float32(logit))))
    py, px = np.mgrid[0:H, 0:W]
    a = np.minimum(0.99, sigma * np.exp(-((px - cam.cx) ** 2 + (py - cam.cy) ** 2) / (2 * v)))
    a = np.where(a >= 1 / 255, a, 0.0) ** 2
    for edge in (cam.cx - 2.3, cam.cx + 0.5, cam.cx + 4.0):
        half = np.array([[edge - 500, -500], [edge, -500], [edge, 600], [edge - 500, 600]])
        c = mlp.rendered_coverage(sc, cam, half, np.zeros(1))[0]
        assert c == pytest.approx(a[px < edge].sum() / a.sum(), rel=1e-12)
    # a region the Gaussian never reaches, and one containing it all
    far = np.array([[1000, 1000], [1100, 1000], [1100, 1100], [1000, 1100]], np.float64)
    assert mlp.rendered_coverage(sc, cam, far, np.zeros(1))[0] == 0.0
    box = np.array([[-10, -10], [60, -10], [60, 60], [-10, 60]], np.float64)
    assert mlp.rendered_coverage(sc, cam, box, np.zeros(1))[0] == pytest.approx(1.0, rel=1e-14)
    # a Gaussian that reaches no pixel takes its plain bit
    off = np.array([[0.0], [0.0], [-5.0]], np.float32)   # behind the camera
    sc2 = sg.Scene(off, sc.log_scale, sc.quat, sc.opacity_logit, sc.sh)
    assert mlp.rendered_coverage(sc2, cam, box, np.ones(1))[0] == 1.0


def test_decisions_truth_table():
    o = np.array([[4.0, 0, 0, 0], [-4.0, 0, 0, 0], [0.1, 2, 2, 2], [4.0, 0, 0, 0]])
    plain = np.array([0, 1, 1, 1], np.uint8)
    valid = np.array([True, True, True, False])
    sel, w, fb = mlp.decisions(o, plain, valid, delta=0.2)
    np.testing.assert_array_equal(fb, [False, False, True, False])
    np.testing.assert_array_equal(sel, [1, 0, 1, 1])
    np.testing.assert_allclose(w[0], 0.5)
    np.testing.assert_allclose(w[2], 1.0)
    np.testing.assert_allclose(w[3], 1.0)


def _f32_forward(theta, X, order, full=False):
    """A float32 implementation rounding at the oracle's points: bf16
    operands, float32 sums over the inputs in the given order, the
    Abramowitz-Stegun 26.2.17 GELU in float32 (full: every intermediate)."""
    P = mlp.unpack(theta)
    f32 = np.float32

    def layer(x, W, b):
        x = x.astype(f32)
        W = W.astype(f32)
        acc = np.broadcast_to(b.astype(f32), (x.shape[0], W.shape[1])).copy()
        for k in order[:W.shape[0]]:
            acc = (acc + x[:, k:k + 1] * W[k:k + 1, :]).astype(f32)
        return acc

    def gelu32(z):
        a = np.abs(z).astype(f32)
        t = (f32(1) / (f32(0.2316419) * a + f32(1))).astype(f32)
        p = t * f32(0.5307027) + f32(-0.72657603)
        p = t * p + f32(0.7107069)
        p = t * p + f32(-0.14224836)
        p = t * p + f32(0.1274148)
        e = np.exp2((f32(-0.7213475) * a) * a).astype(f32)
        q = (e * (p * t)).astype(f32)
        return (z * np.where(z >= 0, f32(1) - q, q)).astype(f32)

    x = mlp.bf16(X)
    z1 = layer(x, mlp.bf16(P["W1"]), P["b1"])
    h1 = mlp.bf16(gelu32(z1).astype(np.float64))
    z2 = layer(h1, mlp.bf16(P["W2"]), P["b2"])
    h2 = mlp.bf16(gelu32(z2).astype(np.float64))
    o = layer(h2, mlp.bf16(P["W3"]), P["b3"])
    if full:
        return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, o=o)
    return o.astype(np.float64)


def test_forward_bound_covers_a_float32_implementation():
    """Every output of a float32 implementation (reverse summation order,
    the A&S GELU) lies within forward_bound of the FP64 oracle; a bound
    without the activations' rounding flips does not, so the flip term is
    exercised."""
    rng = np.random.default_rng(3)
    n = 3000
    X = rng.normal(0, 1.0, (n, 64))
    X[:, 59:] = 0.0
    for seed, scale in ((1, 1.0), (2, 3.0)):
        theta = sg.mlp_init(seed).astype(np.float64) * scale
        f, bound = mlp.forward_bound(theta, X)
        o32 = _f32_forward(theta, X, order=list(range(63, -1, -1)))
        err = np.abs(o32 - f["o"])
        assert np.all(err <= bound), (err / bound).max()
        # without the flip term the bound is the accumulation alone
        P = mlp.unpack(theta)
        g = mlp._gamma(65)
        acc_only = g * ((np.abs(f["h2"])) @ np.abs(mlp.bf16(P["W3"])) + np.abs(P["b3"]))
        assert np.any(err > acc_only)


def _f32_grad(theta, X, sel, cov, B, block=128):
    """The backward of a float32 implementation rounding at loss_grad's
    points: _f32_forward, float32 sigmoid and GELU' (erf), bf16 dz3, dz2,
    dz1, products over the hidden units summed in reverse order, and the
    rows summed in float32 block by block (rows in order within a block of
    128, then the blocks in order)."""
    import scipy.special as sps
    f32 = np.float32
    P = mlp.unpack(theta)
    fw = _f32_forward(theta, X, order=list(range(63, -1, -1)), full=True)
    o = fw["o"].astype(f32)
    p = (f32(1) / (f32(1) + np.exp(-o))).astype(f32)
    inv_b = f32(1.0 / B)
    s_ = np.asarray(sel, f32)
    c_ = np.asarray(cov, f32)[:, None]
    d3 = np.zeros_like(o)
    d3[:, 0] = (p[:, 0] - s_) * inv_b
    d3[:, 1:] = ((f32(2) * (p[:, 1:] - c_)) * p[:, 1:] * (f32(1) - p[:, 1:])) * inv_b

    def ggrad(z):
        z = z.astype(f32)
        e = sps.erf(z * f32(0.70710677)).astype(f32)
        return (f32(0.5) * (f32(1) + e) + z * np.exp(f32(-0.5) * z * z) * f32(0.3989423)).astype(f32)

    def back(D, W):          # D W^T, float32, the hidden units summed in reverse order
        D = D.astype(f32)
        W = W.astype(f32)
        acc = np.zeros((D.shape[0], W.shape[0]), f32)
        for k in range(W.shape[1] - 1, -1, -1):
            acc = (acc + D[:, k:k + 1] * W[:, k][None, :]).astype(f32)
        return acc

    def rowsum(A, Dm):       # A^T Dm, float32, by blocks of rows
        A = A.astype(f32)
        Dm = Dm.astype(f32)
        total = np.zeros((A.shape[1], Dm.shape[1]), f32)
        for b0 in range(0, len(A), block):
            acc = np.zeros_like(total)
            for r in range(b0, min(b0 + block, len(A))):
                acc = (acc + A[r][:, None] * Dm[r][None, :]).astype(f32)
            total = (total + acc).astype(f32)
        return total

    def colsum(Dm):
        return rowsum(np.ones((len(Dm), 1)), Dm)[0]

    d3r = mlp.bf16(d3.astype(np.float64))
    dz2 = back(d3r, mlp.bf16(P["W3"])) * ggrad(fw["z2"])
    dz2r = mlp.bf16(dz2.astype(np.float64))
    dz1 = back(dz2r, mlp.bf16(P["W2"])) * ggrad(fw["z1"])
    dz1r = mlp.bf16(dz1.astype(np.float64))
    g = dict(W3=rowsum(fw["h2"], d3r), b3=colsum(d3), W2=rowsum(fw["h1"], dz2r), b2=colsum(dz2),
             W1=rowsum(fw["x"], dz1r), b1=colsum(dz1))
    return mlp.pack(g)


@pytest.mark.parametrize("scale", [1.0, 3.0])
def test_grad_bound_covers_a_float32_implementation(scale, monkeypatch):
    """Every gradient element of a float32 backward (other summation orders,
    float32 sigmoid and GELU') lies within grad_bound of the FP64 oracle and
    the bound is far below the gradient's scale; with the bf16 flips taken
    out of the bound (no spread beyond the value's own rounding) the same
    float32 backward falls outside it, so those terms are exercised."""
    rng = np.random.default_rng(11)
    n = 2000
    X = rng.normal(0, 1.0, (n, 64))
    X[:, 59:] = 0.0
    sel = (rng.random(n) < 0.4).astype(np.float64)
    cov = rng.random(n)
    theta = sg.mlp_init(4).astype(np.float64) * scale
    depth = 128 + (n + 127) // 128 + 2      # _f32_grad's blocks of 128 rows
    for B in (n, n + 7):
        g32 = _f32_grad(theta, X, sel, cov, B)
        for d in (None, depth):
            loss, g, bound = mlp.grad_bound(theta, X, sel, cov, batch=B, depth=d)
            err = np.abs(g32 - g)
            assert np.all(err <= bound), (err / bound).max()
        # most of the bound is the chance of bf16 flips, far below the gradient
        assert np.median(bound) <= 0.05 * np.abs(g).max()
    monkeypatch.setattr(mlp, "_bf16_spread", lambda v, d: np.zeros_like(np.asarray(v, float)))
    _, g, no_flips = mlp.grad_bound(theta, X, sel, cov, batch=n, depth=depth)
    assert np.any(np.abs(_f32_grad(theta, X, sel, cov, n) - g) > no_flips)


def _f32_features(scene, cam, xy):
    """Features 0-9 of a float32 implementation: the view transform, the
    projection, the radial frame, the eigen-decomposition and the logs in
    float32 (numpy rounds each step), from the oracle's 2D covariance
    rounded to float32."""
    import oracle as O
    f32 = np.float32
    x = np.asarray(scene.xyz, f32)
    V = np.asarray(cam.world_to_view, f32).reshape(3, 4)
    t = [(V[i, 0] * x[0] + V[i, 1] * x[1] + V[i, 2] * x[2] + V[i, 3]).astype(f32) for i in range(3)]
    tz = t[2]
    valid = tz > f32(cam.z_near)
    tzs = np.where(valid, tz, f32(1))
    iz = (f32(1) / tzs).astype(f32)
    u = (f32(cam.fx) * (t[0] * iz) + f32(cam.cx)).astype(f32)
    v = (f32(cam.fy) * (t[1] * iz) + f32(cam.cy)).astype(f32)
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    cen = xy.mean(0).astype(f32)
    qx, qy = (u - cen[0]).astype(f32), (v - cen[1]).astype(f32)
    lam = np.full(len(u), np.inf, f32)
    for i in range(len(xy)):
        ax, ay = (xy[i - 1] - xy.mean(0)).astype(f32)
        ex, ey = (xy[i] - xy[i - 1]).astype(f32)
        den = (qx * ey - qy * ex).astype(f32)
        with np.errstate(divide="ignore", invalid="ignore"):
            idn = (f32(1) / den).astype(f32)
            l = ((ax * ey - ay * ex) * idn).astype(f32)
            sp = ((ax * qy - ay * qx) * idn).astype(f32)
        ok = (den != 0) & (l > 0) & (sp >= 0) & (sp <= 1) & (l < lam)
        lam = np.where(ok, l, lam)
    qn = np.sqrt(qx * qx + qy * qy).astype(f32)
    mean_r = f32(np.sqrt(((xy - xy.mean(0)) ** 2).sum(1)).mean())
    rho = np.where(np.isfinite(lam) & (qn > 0), lam * qn, mean_r).astype(f32)
    sp_ = O.preprocess(scene, cam)
    a, b, c = (sp_["cov2d"][k::3].astype(f32) for k in range(3))
    a, b, c = np.where(valid, a, f32(1)), np.where(valid, b, f32(0)), np.where(valid, c, f32(1))
    iq = np.where(qn > 0, f32(1) / np.where(qn > 0, qn, f32(1)), f32(0)).astype(f32)
    ux = np.where(qn > 0, qx * iq, f32(1)).astype(f32)
    uy = np.where(qn > 0, qy * iq, f32(0)).astype(f32)
    mid = (f32(0.5) * (a + c)).astype(f32)
    rad = np.sqrt(f32(0.25) * (a - c) * (a - c) + b * b).astype(f32)
    irad = np.where(rad > 0, f32(1) / np.where(rad > 0, rad, f32(1)), f32(0)).astype(f32)
    c2p = np.where(rad > 0, f32(0.5) * (a - c) * irad, f32(1)).astype(f32)
    s2p = np.where(rad > 0, b * irad, f32(0)).astype(f32)
    c2q, s2q = (ux * ux - uy * uy).astype(f32), (f32(2) * ux * uy).astype(f32)
    sr = np.sqrt(a * ux * ux + f32(2) * b * ux * uy + c * uy * uy).astype(f32)
    lr = np.log(rho).astype(f32)
    G = np.zeros((len(u), 10), f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        G[:, 0] = (qx / rho)
        G[:, 1] = (qy / rho)
        G[:, 2] = np.log(tzs * rho * (f32(1) / f32(cam.fx)))
        G[:, 3] = f32(0.5) * np.log(mid + rad) - lr
        G[:, 4] = f32(0.5) * np.log(mid - rad) - lr
        G[:, 5] = np.log(sr) - lr
        G[:, 6] = c2p * c2q + s2p * s2q
        G[:, 7] = s2p * c2q - c2p * s2q
        G[:, 8] = np.clip((rho - qn) * (f32(1) / sr), f32(-8), f32(8))
    G[:, :9] = np.where(valid[:, None], G[:, :9], f32(0))
    ls = np.asarray(scene.log_scale, f32)
    G[:, 9] = ((ls[0] + ls[1] + ls[2]) * f32(1.0 / 3.0)).astype(f32)
    return G.astype(np.float64), valid


def test_feature_bound_covers_a_float32_implementation():
    """Every feature of a float32 implementation, rounded to bf16, lies in
    the bf16 interval feature_bound gives; the bound is a small fraction of
    a bf16 step except for the orientation of near-isotropic footprints;
    without the input-error terms it is exceeded."""
    from paper_2511_18441_b300 import scenegen as sgen
    w = sgen.paper_scale_workload(n=20000, seed=7, width=320, height=240)
    reg = sgen.random_polygons(1, 320, 240, 11)[0]
    F, valid, E = mlp.feature_bound(w.scene, w.camera, reg.xy)
    G, v32 = _f32_features(w.scene, w.camera, reg.xy)
    assert np.array_equal(valid, v32)
    ok = mlp.bf16_within(mlp.bf16(G), F[:, :10], E[:, :10])
    assert ok.all(), np.argwhere(~ok)[:5]
    step = np.maximum(np.abs(F[valid, :6]), 1e-3) * 2.0 ** -8
    assert np.median(E[valid, :6] / step) < 0.02
    # the float32 result does move by more than its own roundings would allow
    loose = np.abs(G[:, :9] - F[:, :9]) > 64 * 2.0 ** -24 * (1 + np.abs(F[:, :9]))
    assert loose[valid].any()


def _f32_weight_sums(sp, off, ids, weight, width, height, power):
    """Sums of weight (alpha T)^power per splat from a float32 walk (as
    f32_color_grad of the gradient pins, one channel)."""
    f32 = np.float32
    n = sp["n"]
    u, v = sp["u"].astype(f32), sp["v"].astype(f32)
    A, B, Cc = (sp["conic"][k::3].astype(f32) for k in range(3))
    sig = sp["opacity"].astype(f32)
    valid = sp["valid"].astype(bool)
    out = np.zeros(n, f32)
    wgt = np.asarray(weight, f32).reshape(height, width)
    tx = (width + 15) // 16
    for t in range(len(off) - 1):
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        xs, ys = np.meshgrid(np.arange(x0, min(x0 + 16, width)), np.arange(y0, min(y0 + 16, height)))
        xs, ys = xs.ravel().astype(f32), ys.ravel().astype(f32)
        gp = wgt[ys.astype(int), xs.astype(int)]
        T = np.ones(len(xs), f32)
        live = np.ones(len(xs), bool)
        for k in range(off[t], off[t + 1]):
            i = int(ids[k])
            if not valid[i]:
                continue
            dx, dy = xs - u[i], ys - v[i]
            p = np.minimum((f32(-0.5) * (A[i] * dx * dx + Cc[i] * dy * dy) - B[i] * dx * dy).astype(f32),
                           f32(0))
            al = np.minimum(f32(0.99), (sig[i] * np.exp(p)).astype(f32))
            take = live & (al >= f32(1.0 / 255.0))
            nT = (T * (f32(1) - al)).astype(f32)
            stop = take & (nT < f32(1e-4))
            live &= ~stop
            take &= ~stop
            wv = (al * T).astype(f32)
            for val in (gp[take] * wv[take] ** power).astype(f32):
                out[i] = f32(out[i] + val)
            T = np.where(take, nT, T)
    return out.astype(np.float64)


def test_coverage_bound_covers_a_float32_walk():
    """The tint-weight label of a float32 walk (sums of (alpha T)^2 inside
    the polygon and over all pixels, then their ratio) lies in the interval
    coverage_bound gives, for every splat."""
    import oracle as O
    from paper_2511_18441_b300 import scenegen as sgen
    w = sgen.paper_scale_workload(n=4000, seed=5, width=96, height=64)
    reg = sgen.random_polygons(1, 96, 64, 3)[0]
    F, valid, sel, cov = mlp.features_and_labels(w.scene, w.camera, reg.xy)
    c2, lo, hi = mlp.coverage_bound(w.scene, w.camera, reg.xy, sel)
    np.testing.assert_array_equal(c2, cov)
    sp = O.preprocess(w.scene, w.camera)
    off, ids = O.tile_lists(sp, O.depth_order(sp), 6, 4)
    py, px = np.mgrid[0:64, 0:96]
    inside = mlp.point_in_polygon(px.ravel().astype(np.float64), py.ravel().astype(np.float64),
                                  reg.xy).astype(np.float64)
    num = _f32_weight_sums(sp, off, ids, inside, 96, 64, 2)
    den = _f32_weight_sums(sp, off, ids, np.ones(96 * 64), 96, 64, 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = np.minimum(num.astype(np.float32) / den.astype(np.float32), 1.0)
    lab = np.where(den > 0, ratio, sel.astype(np.float64))
    ok = (lab >= lo) & (lab <= hi)
    assert ok.all(), (lab[~ok][:5], lo[~ok][:5], hi[~ok][:5])
    reach = den > 0
    assert reach.sum() > 500 and np.median((hi - lo)[reach]) < 1e-3
