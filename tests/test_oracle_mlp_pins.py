"""Pins of the learned-selection oracle (oracle/mlp.py) against facts fixed
outside it: finite differences of its own loss (FP64 path), torch's bfloat16
conversion, closed forms of GELU, the radial frame and the Gauss-Hermite
rule, and the plain selection. ReCoGS (arXiv 2511.18441) names the leak of
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


def test_gauss_hermite_rule_moments():
    x, w = mlp.hermite_rule()
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(np.sort(x), -np.sort(x)[::-1], atol=1e-15)
    # a 5-point rule integrates polynomials up to degree 9 exactly (N(0,1) moments)
    for k, m in ((2, 1.0), (4, 3.0), (6, 15.0), (8, 105.0)):
        assert (w * x ** k).sum() == pytest.approx(m, rel=1e-12)


def test_quadrature_points_reproduce_mean_and_covariance():
    """The rule integrates quadratics exactly: the weighted points have the
    Gaussian's mean and covariance (this fixes the Cholesky factor)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        A = rng.normal(size=(2, 2))
        S = A @ A.T + 0.3 * np.eye(2)
        mu = rng.normal(0, 50, 2)
        pu, pv, w = mlp.quadrature_points(mu[0], mu[1], S[0, 0], S[0, 1], S[1, 1])
        m = np.array([(w * pu).sum(), (w * pv).sum()])
        np.testing.assert_allclose(m, mu, rtol=1e-12, atol=1e-9)
        d = np.stack([pu - mu[0], pv - mu[1]])
        C = (w * d) @ d.T
        np.testing.assert_allclose(C, S, rtol=1e-10, atol=1e-10)


def small_scene(n=300, seed=3):
    w = sg.tiny_workload(n=n, seed=seed, width=64, height=64)
    return w.scene, w.camera


def test_features_layout_and_plain_label():
    scene, cam = small_scene()
    xy = sg.polygon_region(64, 64, 12, 0.2, 5).xy
    F, valid, sel, cov = mlp.features_and_labels(scene, cam, xy)
    n = scene.n
    np.testing.assert_array_equal(F[:, 3:6], scene.log_scale.T.astype(np.float64))
    np.testing.assert_allclose((F[:, 6:10] ** 2).sum(1), 1.0, rtol=1e-12)
    np.testing.assert_array_equal(F[:, 10], scene.opacity_logit.astype(np.float64))
    np.testing.assert_array_equal(F[:, 11:59], scene.sh.reshape(48, n).T.astype(np.float64))
    assert not F[:, 59:].any()
    edit = sg.Edit(sg.Region("polygon", xy), np.eye(3, dtype=np.float32), cam)
    ref, _ = oracle.select(scene, edit, cam)
    np.testing.assert_array_equal(sel, ref)
    assert valid.all() and 0.05 < sel.mean() < 0.95
    assert ((cov >= 0) & (cov <= 1 + 1e-12)).all()
    # centre inside the polygon frame <=> plain selection, for a star-shaped polygon
    r = np.hypot(F[:, 0], F[:, 1])
    far = np.abs(r - 1) > 1e-9
    np.testing.assert_array_equal((r < 1)[far], sel.astype(bool)[far])


def test_coverage_of_tiny_and_straddling_gaussians():
    """Far inside -> 1, far outside -> 0; a splat cut by a straight edge at
    offset d (in units of its standard deviation along the normal) covers
    the weight of the 1D rule's nodes on the inside of the edge."""
    cam = sg.axis_camera(101, 101, 60.0, 3.0)
    s = 0.004
    mus = [(0, 0, 0), (2.0, 2.0, 0)]
    sc = sg.Scene(np.array(mus, np.float32).T.copy(), np.full((3, 2), math.log(s), np.float32),
                  np.tile(np.array([[1.0], [0], [0], [0]], np.float32), 2),
                  np.zeros(2, np.float32), np.zeros((16, 3, 2), np.float32))
    box = np.array([[10, 10], [90, 10], [90, 90], [10, 90]], np.float64)
    F, valid, sel, cov = mlp.features_and_labels(sc, cam, box)
    assert cov[0] == pytest.approx(1.0, rel=1e-12) and cov[1] == 0.0
    # a vertical edge at u = cx + d sigma: inside where u + sigma x < cx + d sigma
    sp = oracle.preprocess(sc, cam)
    sigma = math.sqrt(sp["cov2d"][0])
    x, w = mlp.hermite_rule()
    for d in (-1.7, -0.3, 0.4, 1.1):
        edge = cam.cx + d * sigma
        half = np.array([[edge - 500, -500], [edge, -500], [edge, 600], [edge - 500, 600]])
        c = mlp.features_and_labels(sc, cam, half)[3][0]
        assert c == pytest.approx(w[x < d].sum(), abs=1e-12)


def test_decisions_truth_table():
    o = np.array([[4.0, 0, 0, 0], [-4.0, 0, 0, 0], [0.1, 2, 2, 2], [4.0, 0, 0, 0]])
    plain = np.array([0, 1, 1, 1], np.uint8)
    exact = np.array([0.2, 0.3, 0.4, 0.5])
    valid = np.array([True, True, True, False])
    sel, w, fb = mlp.decisions(o, plain, exact, valid, delta=0.2)
    np.testing.assert_array_equal(fb, [False, False, True, False])
    np.testing.assert_array_equal(sel, [1, 0, 1, 1])
    np.testing.assert_allclose(w[0], 0.5)
    np.testing.assert_allclose(w[2], 0.4)
    np.testing.assert_allclose(w[3], 1.0)
