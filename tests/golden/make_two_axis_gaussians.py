"""Writes two_axis_gaussians_16x16.txt: a worked example of Eq. 1-3 in
closed form, computed here without the oracle.

Two isotropic Gaussians on the optical axis of a camera at (0, 0, -3) looking
along +z (view rotation the identity), 16x16 pixels, vertical field of view
60 degrees, background (0.1, 0.2, 0.3). For an isotropic Gaussian of scale s
at view depth Z on the axis the Jacobian of the projection is diag(f/Z, f/Z)
(its third column vanishes at x = y = 0), so the projected covariance with
the 0.3 pixel^2 dilation is v I, v = (f s / Z)^2 + 0.3, centred on the
principal point (Eq. 1). Seen along +z only the m = 0 real SH terms are
non-zero, Y_l0 = sqrt((2l + 1) / (4 pi)), so the colour is
max(sum_l C_l0 Y_l0 + 0.5, 0) (Eq. 2). Pixel (x, y) composites the nearer
Gaussian first (Eq. 3): alpha = min(0.99, sigma exp(-|d|^2 / (2 v))), a
Gaussian with alpha < 1/255 is skipped, and
C = sum_i c_i alpha_i T_i + T bg, T_i = prod_{j<i} (1 - alpha_j).

Scene values are float32 (as stored); the arithmetic is float64.
Run: python tests/golden/make_two_axis_gaussians.py
"""
import math
import os

import numpy as np

W = H = 16
FOVY = 60.0
DIST = 3.0
BG = (0.1, 0.2, 0.3)
# (z, scale, opacity logit): view depths 2.5 and 3.7
SPLATS = ((-0.5, 0.6, 0.4), (0.7, 0.9, 1.2))
SEED = 5


def main():
    rng = np.random.default_rng(SEED)
    sh = rng.normal(0, 0.3, size=(len(SPLATS), 16, 3)).astype(np.float32)
    f = H / (2.0 * math.tan(math.radians(FOVY) / 2.0))
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    gs = []
    for (z, s, logit), c in zip(SPLATS, sh):
        z32 = float(np.float32(z))
        s32 = math.exp(float(np.float32(math.log(s))))
        l32 = float(np.float32(logit))
        Z = z32 + DIST
        v = (f * s32 / Z) ** 2 + 0.3
        sigma = 1.0 / (1.0 + math.exp(-l32))
        col = [max(sum(float(c[l * l + l, ch]) * math.sqrt((2 * l + 1) / (4 * math.pi))
                       for l in range(4)) + 0.5, 0.0) for ch in range(3)]
        gs.append((Z, v, sigma, col))
    gs.sort(key=lambda g: g[0])
    rows = []
    for y in range(H):
        for x in range(W):
            d2 = (x - cx) ** 2 + (y - cy) ** 2
            T, C = 1.0, [0.0, 0.0, 0.0]
            for Z, v, sigma, col in gs:
                a = min(0.99, sigma * math.exp(-d2 / (2.0 * v)))
                # no decision may sit near a threshold
                assert abs(a - 1 / 255) > 1e-3 / 255
                if a < 1 / 255:
                    continue
                assert T * (1 - a) >= 1e-4
                for ch in range(3):
                    C[ch] += col[ch] * a * T
                T *= 1 - a
            rows.append((x, y, C[0] + T * BG[0], C[1] + T * BG[1], C[2] + T * BG[2], T))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_axis_gaussians_16x16.txt")
    with open(out, "w") as fh:
        fh.write("# Two on-axis isotropic Gaussians, closed form of Eq. 1-3 (ReCoGS, arXiv\n"
                 "# 2511.18441, Sec. 3.1); written by make_two_axis_gaussians.py, see there.\n")
        fh.write(f"# camera: {W}x{H}, fovy {FOVY} deg, at (0, 0, -{DIST}) looking along +z\n")
        fh.write(f"bg {BG[0]!r} {BG[1]!r} {BG[2]!r}\n")
        for (z, s, logit), c in zip(SPLATS, sh):
            fh.write(f"splat {z!r} {s!r} {logit!r} " + " ".join(repr(float(q)) for q in c.ravel())
                     + "\n")
        fh.write("# pixel x y r g b T\n")
        for r in rows:
            fh.write("pixel %d %d %.17g %.17g %.17g %.17g\n" % r)


if __name__ == "__main__":
    main()
