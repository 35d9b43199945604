"""Readers of the stored fixtures under tests/golden/ (no arithmetic of the
method here: parsing and scene assembly only)."""
import math
import os

import numpy as np

from paper_2511_18441_b300 import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def two_axis_gaussians():
    """(scene, camera, bg, rgb [H, W, 3], T [H, W]) of
    two_axis_gaussians_16x16.txt."""
    splats, px = [], []
    bg = None
    with open(os.path.join(GOLDEN, "two_axis_gaussians_16x16.txt")) as f:
        for line in f:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "bg":
                bg = tuple(float(q) for q in p[1:4])
            elif p[0] == "splat":
                splats.append([float(q) for q in p[1:]])
            elif p[0] == "pixel":
                px.append([float(q) for q in p[1:]])
    n = len(splats)
    xyz = np.zeros((3, n), np.float32)
    log_scale = np.zeros((3, n), np.float32)
    quat = np.zeros((4, n), np.float32)
    quat[0] = 1.0
    logit = np.zeros(n, np.float32)
    sh = np.zeros((16, 3, n), np.float32)
    for i, s in enumerate(splats):
        xyz[2, i] = s[0]
        log_scale[:, i] = math.log(s[1])
        logit[i] = s[2]
        sh[:, :, i] = np.asarray(s[3:], np.float32).reshape(16, 3)
    scene = sg.Scene(xyz, log_scale, quat, logit, sh)
    cam = sg.axis_camera(16, 16, 60.0, 3.0)
    px = np.asarray(px)
    rgb = np.zeros((16, 16, 3))
    T = np.zeros((16, 16))
    for x, y, r, g, b, t in px:
        rgb[int(y), int(x)] = (r, g, b)
        T[int(y), int(x)] = t
    return scene, cam, bg, rgb, T
