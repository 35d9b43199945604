"""Seeded input generator: determinism, shapes and the stated recipe."""
import math

import numpy as np
import pytest

from paper_2511_18441_b300 import scenegen as sg


def test_deterministic_and_shaped():
    a = sg.tiny_workload()
    b = sg.tiny_workload()
    for f in ("xyz", "log_scale", "quat", "opacity_logit", "sh"):
        x, y = getattr(a.scene, f), getattr(b.scene, f)
        assert x.dtype == np.float32 and x.flags.c_contiguous
        assert np.array_equal(x, y)
    s = a.scene
    assert s.xyz.shape == (3, 10000) and s.sh.shape == (16, 3, 10000)
    assert s.quat.shape == (4, 10000) and s.opacity_logit.shape == (10000,)


def test_recipe_statistics():
    s = sg.make_scene(200_000, 5, 5.0, 40, (2.0, 5.0), 20, (2.0, 5.0))
    assert s.log_scale.mean() == pytest.approx(-4.5, abs=0.01)
    assert s.log_scale.std() == pytest.approx(0.5, abs=0.01)
    assert s.opacity_logit.std() == pytest.approx(1.5, abs=0.02)
    np.testing.assert_allclose(np.linalg.norm(s.quat, axis=0), 1.0, atol=1e-6)
    assert s.sh[1:].std() == pytest.approx(0.03, abs=0.001)
    assert np.abs(s.xyz).max() < 5.0 + 5.0 + 0.1


def test_polygon_area_and_centre():
    r = sg.polygon_region(1920, 1080, 12, 0.15, 1)
    assert r.xy.shape == (12, 2)
    assert sg.shoelace_area(r.xy) == pytest.approx(0.15 * 1920 * 1080, rel=1e-5)
    assert r.xy.mean(0) == pytest.approx([959.5, 539.5], abs=200)


def test_hue_matrix_keeps_grey():
    M = sg.hue_rotation_matrix(90.0).astype(np.float64)
    np.testing.assert_allclose(M @ np.ones(3), np.ones(3), atol=1e-6)
    np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-6)


def test_axis_camera_is_identity_rotation():
    c = sg.axis_camera(1920, 1080, 60.0, 14.0)
    np.testing.assert_allclose(c.world_to_view[:, :3], np.eye(3), atol=1e-7)
    np.testing.assert_allclose(c.world_to_view[:, 3], [0, 0, 14.0])
    assert c.fy == pytest.approx(1080 / (2 * math.tan(math.radians(30))))
    assert c.cx == 959.5 and c.cy == 539.5


def test_half_precision_round_trip():
    rng = np.random.default_rng(0)
    x = rng.normal(size=1000).astype(np.float32)
    for kind, rel in (("f16", 2 ** -11), ("bf16", 2 ** -8)):
        y = sg.from_half(sg.to_half(x, kind), kind)
        assert np.all(np.abs(y - x) <= rel * np.abs(x) + 1e-7)
