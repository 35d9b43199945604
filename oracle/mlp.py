"""FP64 oracle of the learned selection MLP (numpy).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the product
package; it imports nothing from the product package.

The paper names the leak of its selection as a limitation (Sec. 6: a
Gaussian larger than the selection is recoloured as a whole or not at all).
The learned variant predicts, per Gaussian, the plain selection bit (a
logit) and its tint weight (one per RGB channel, the "tint residual"), from
59 features that express the splat in the selection view:

  0, 1  the centre, (u, v) - c, divided by the distance rho from the
        polygon's vertex centroid c to the polygon boundary along that
        direction (a star-shaped polygon maps onto the unit disc)
  2     ln(t_z rho / f_x)
  3, 4  ln(sigma_1 / rho), ln(sigma_2 / rho): standard deviations of the
        projected 2D Gaussian (the dilated Sigma' of the render) along its
        axes
  5     ln(sigma_r / rho): its standard deviation along the radial
        direction q = (u, v) - c
  6, 7  cos 2 theta, sin 2 theta: the major axis' angle to q
  8     (rho - |q|) / sigma_r, clamped to [-8, 8]: the distance to the
        boundary along q in radial standard deviations (positive inside)
  9     the mean of the three log-scales; 10 the opacity logit
  11-58 the 48 SH coefficients ([16][3] order)
  59-63 zero padding (K = 64)

Tint-weight label: the least-squares per-Gaussian weight of the selection
view's render, sum over inside pixels of (alpha_i T_i)^2 / sum over all
pixels (Eq. 3's contributions; pixels inside by the plain even-odd test at
their centres); a Gaussian that reaches no pixel takes its plain bit. For a
Gaussian whose colour error does not overlap others', recolouring it by
weight w changes the error at pixel p by (w - 1[p inside]) alpha_i T_i
(t - 1) c_i, whose sum of squares this weight minimises. Splats with
t_z <= z_near are outside the learned domain (the plain test decides them).

Network (BF16 weights, FP32 accumulation): z1 = x W1 + b1, h1 = GELU(z1),
z2 = h1 W2 + b2, h2 = GELU(z2), o = h2 W3 + b3 (o0 = selection logit,
o1..o3 = coverage logits), GELU(z) = z Phi(z) with the exact normal CDF.
The inputs of every product (features, weights, h1, h2 and the backward's
dz3, dz2, dz1) are rounded to bfloat16 (round to nearest even) and products
are summed in wide precision; with rnd=False the same network runs in FP64
throughout (used by the finite-difference pins).

Loss per sample: BCE(o0, sel) + sum_c (sigmoid(o_c) - coverage)^2, mean
over the batch.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sps

import oracle as _o

N_IN = 59
K = 64
H = 64
N_OUT = 4
# parameter vector: W1 [64][64] (input-major), b1 [64], W2 [64][64], b2 [64],
# W3 [64][4], b3 [4]
SHAPES = (("W1", (K, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, N_OUT)),
          ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), as float64 values."""
    a = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def gelu(z):
    return z * 0.5 * (1.0 + sps.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + sps.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


# ---------------------------------------------------------------------------
# features and labels

def point_in_polygon(u, v, xy):
    """Even-odd rule, vectorised over points (same convention as the plain
    selection: an edge counts when exactly one end is strictly above v)."""
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    inside = np.zeros(np.shape(u), bool)
    n = len(xy)
    for i in range(n):
        xi, yi = xy[i]
        xj, yj = xy[i - 1]
        cond = (yi > v) != (yj > v)
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = xi + (v - yi) * (xj - xi) / (yj - yi)
        inside ^= cond & (u < xc)
    return inside


def radial_frame(u, v, xy):
    """(q / rho, rho): q = (u, v) - centroid, rho = distance from the vertex
    centroid to the boundary along q (the nearest edge crossing of the ray)."""
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    c = xy.mean(0)
    mean_r = np.sqrt(((xy - c) ** 2).sum(1)).mean()
    qx, qy = u - c[0], v - c[1]
    lam = np.full(np.shape(u), np.inf)
    n = len(xy)
    for i in range(n):
        ax, ay = xy[i - 1] - c
        ex, ey = xy[i] - xy[i - 1]
        den = qx * ey - qy * ex
        with np.errstate(divide="ignore", invalid="ignore"):
            l = (ax * ey - ay * ex) / den
            s = (ax * qy - ay * qx) / den
        ok = (den != 0) & (l > 0) & (s >= 0) & (s <= 1)
        lam = np.where(ok & (l < lam), l, lam)
    qn = np.sqrt(qx * qx + qy * qy)
    with np.errstate(invalid="ignore"):
        rho = np.where(np.isfinite(lam) & (qn > 0), lam * qn, mean_r)
    return qx / rho, qy / rho, rho


def _view_centre(scene, cam):
    """View-space centre t (3 x n), projected centre (u, v) and validity."""
    xyz = np.asarray(scene.xyz, np.float32).astype(np.float64)
    V = np.asarray(cam.world_to_view, np.float32).astype(np.float64).reshape(3, 4)
    t = V[:, :3] @ xyz + V[:, 3:4]
    tz = t[2]
    valid = tz > float(np.float32(cam.z_near))
    with np.errstate(divide="ignore", invalid="ignore"):
        u = float(np.float32(cam.fx)) * t[0] / tz + float(np.float32(cam.cx))
        v = float(np.float32(cam.fy)) * t[1] / tz + float(np.float32(cam.cy))
    return xyz, V, t, np.where(valid, u, 0.0), np.where(valid, v, 0.0), valid


def _geometry(u, v, tz, a, b, c, valid, region_xy, fx):
    """Features 0-8 (the splat in the selection view, see the header) from
    the projected centre, the view depth and the dilated 2D covariance,
    with the intermediate magnitudes a float32 evaluation rounds."""
    un, vn, rho = radial_frame(u, v, region_xy)
    a, b, c = np.where(valid, a, 1.0), np.where(valid, b, 0.0), np.where(valid, c, 1.0)
    cen = np.asarray(region_xy, np.float64).reshape(-1, 2).mean(0)
    qx, qy = u - cen[0], v - cen[1]
    qn = np.sqrt(qx * qx + qy * qy)
    ux = np.where(qn > 0, qx / np.where(qn > 0, qn, 1.0), 1.0)
    uy = np.where(qn > 0, qy / np.where(qn > 0, qn, 1.0), 0.0)
    mid = 0.5 * (a + c)
    rad = np.sqrt(0.25 * (a - c) ** 2 + b * b)
    l1, l2 = mid + rad, mid - rad
    c2p = np.where(rad > 0, 0.5 * (a - c) / np.where(rad > 0, rad, 1.0), 1.0)
    s2p = np.where(rad > 0, b / np.where(rad > 0, rad, 1.0), 0.0)
    c2q, s2q = ux * ux - uy * uy, 2 * ux * uy
    sr = np.sqrt(a * ux * ux + 2 * b * ux * uy + c * uy * uy)
    lr = np.log(rho)
    G = np.zeros((len(u), 9))
    with np.errstate(divide="ignore", invalid="ignore"):
        G[:, 0] = np.where(valid, un, 0.0)
        G[:, 1] = np.where(valid, vn, 0.0)
        G[:, 2] = np.where(valid, np.log(np.where(valid, tz, 1.0) * rho / fx), 0.0)
        G[:, 3] = np.where(valid, 0.5 * np.log(l1) - lr, 0.0)
        G[:, 4] = np.where(valid, 0.5 * np.log(l2) - lr, 0.0)
        G[:, 5] = np.where(valid, np.log(sr) - lr, 0.0)
        G[:, 6] = np.where(valid, c2p * c2q + s2p * s2q, 0.0)
        G[:, 7] = np.where(valid, s2p * c2q - c2p * s2q, 0.0)
        G[:, 8] = np.where(valid, np.clip((rho - qn) / sr, -8.0, 8.0), 0.0)
    mags = dict(rho=rho, qn=qn, mid=mid, rad=rad, l1=l1, l2=l2, sr=sr,
                sq=np.abs(a) * ux * ux + 2 * np.abs(b * ux * uy) + np.abs(c) * uy * uy,
                ac=np.abs(a) + np.abs(b) + np.abs(c))
    return G, mags


def features_and_labels(scene, cam, region_xy):
    """Returns (F [n, 64], valid [n] bool, sel [n] uint8, coverage [n])."""
    n = scene.xyz.shape[1]
    xyz, V, t, uu, vv, valid = _view_centre(scene, cam)
    sp = _o.preprocess(scene, cam)
    a, b, c = sp["cov2d"][0::3], sp["cov2d"][1::3], sp["cov2d"][2::3]
    G, _ = _geometry(uu, vv, t[2], a, b, c, valid, region_xy, float(np.float32(cam.fx)))
    F = np.zeros((n, K))
    F[:, :9] = G
    F[:, 9] = np.asarray(scene.log_scale, np.float32).astype(np.float64).mean(0)
    F[:, 10] = np.asarray(scene.opacity_logit, np.float32)
    F[:, 11:59] = np.asarray(scene.sh, np.float32).reshape(48, n).T
    # labels: the plain selection bit and the rendered coverage
    edit = type("E", (), {})()
    edit.region = type("R", (), {})()
    edit.region.kind = "polygon"
    edit.region.xy = np.asarray(region_xy, np.float64).reshape(-1, 2)
    edit.color_matrix = np.eye(3)
    edit.select_camera = cam
    sel, _ = _o.select(scene, edit, cam)
    cov = rendered_coverage(scene, cam, region_xy, sel)
    return F, valid, sel.astype(np.uint8), cov


def rendered_coverage(scene, cam, region_xy, plain_sel):
    """sum over inside pixels of (alpha_i T_i)^2 / sum over all pixels, from
    the binned FP64 render of the selection view; the plain bit where the
    splat reaches no pixel."""
    sp = _o.preprocess(scene, cam)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    off, ids = _o.tile_lists(sp, _o.depth_order(sp), tx, ty)
    H, W = cam.height, cam.width
    py, px = np.mgrid[0:H, 0:W]
    inside = point_in_polygon(px.ravel().astype(np.float64), py.ravel().astype(np.float64),
                              region_xy).astype(np.float64)
    num = _o.weight_sums(sp, off, ids, inside, 2)
    den = _o.weight_sums(sp, off, ids, np.ones(H * W), 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(den > 0, np.minimum(num / den, 1.0), np.asarray(plain_sel, np.float64))


# A float32 evaluation of the features departs from them through (1) its
# inputs: the view-space centre (three float32 FMAs of the view transform,
# e_t = 4 u32 (sum_k |V_ik x_k| + |V_i3|)), the projected centre (an
# approximate reciprocal of t_z, 2^-22 relative, and two roundings) and the
# dilated 2D covariance (within COV_REL sqrt(a c) per entry, the render's
# margin), carried through the features by central differences of the FP64
# features over each input's error (times 2 for the curvature), and (2) the
# roundings of its own steps, bounded from the magnitudes they act on
# (cancellations in mid - rad, a - c, rho - |q| and the quadratic form), and
# the fast logarithms (LOG_ERR absolute).
U32 = 2.0 ** -24
COV_REL = 1e-5
LOG_ERR = 2e-6


def feature_bound(scene, cam, region_xy):
    """(F, valid, E): the features of features_and_labels and, per element,
    a bound on a float32 implementation's departure from F before its bf16
    rounding (so its bf16 feature lies in [bf16(F - E), bf16(F + E)])."""
    n = scene.xyz.shape[1]
    xyz, V, t, uu, vv, valid = _view_centre(scene, cam)
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    et = 4 * U32 * (np.abs(V[:, :3]) @ np.abs(xyz) + np.abs(V[:, 3:4]))
    tz = np.where(valid, t[2], 1.0)
    rel_iz = et[2] / np.abs(tz) + 2.0 ** -22
    eu = fx * (et[0] / np.abs(tz) + np.abs(t[0] / tz) * rel_iz) + 2 * U32 * (np.abs(uu) + abs(cx))
    ev = fy * (et[1] / np.abs(tz) + np.abs(t[1] / tz) * rel_iz) + 2 * U32 * (np.abs(vv) + abs(cy))
    sp = _o.preprocess(scene, cam)
    a, b, c = sp["cov2d"][0::3], sp["cov2d"][1::3], sp["cov2d"][2::3]
    ecov = COV_REL * np.sqrt(np.abs(np.where(valid, a, 1.0) * np.where(valid, c, 1.0)))
    base = (uu, vv, t[2], a, b, c)
    G, m = _geometry(*base, valid, region_xy, fx)
    E = np.zeros((n, K))
    for k, e in enumerate((eu, ev, et[2], ecov, ecov, ecov)):
        hi = list(base)
        lo = list(base)
        hi[k] = base[k] + e
        lo[k] = base[k] - e
        Gh, _ = _geometry(*hi, valid, region_xy, fx)
        Gl, _ = _geometry(*lo, valid, region_xy, fx)
        E[:, :9] += np.abs(Gh - Gl)       # twice the central difference
    # the float32 steps' own roundings
    with np.errstate(divide="ignore", invalid="ignore"):
        r_eig = 8 * U32 * (m["mid"] + m["rad"])
        E[:, 0] += 8 * U32 * np.abs(G[:, 0])
        E[:, 1] += 8 * U32 * np.abs(G[:, 1])
        E[:, 2] += LOG_ERR + 8 * U32
        E[:, 3] += 2 * LOG_ERR + 0.5 * r_eig / m["l1"]
        E[:, 4] += 2 * LOG_ERR + 0.5 * r_eig / np.where(m["l2"] > 0, m["l2"], np.inf)
        E[:, 5] += 2 * LOG_ERR + 8 * U32 * m["sq"] / (m["sr"] ** 2)
        rot = 16 * U32 * m["ac"] / np.where(m["rad"] > 0, m["rad"], np.inf)
        E[:, 6] += rot + 16 * U32
        E[:, 7] += rot + 16 * U32
        E[:, 8] += 8 * U32 * (m["rho"] + m["qn"]) / m["sr"] + 8 * U32 * np.abs(G[:, 8])
    E[:, :9] = np.where(valid[:, None] & np.isfinite(E[:, :9]), E[:, :9],
                        np.where(valid[:, None], np.inf, 0.0))
    F = np.zeros((n, K))
    F[:, :9] = G
    ls = np.asarray(scene.log_scale, np.float32).astype(np.float64)
    F[:, 9] = ls.mean(0)
    E[:, 9] = 4 * U32 * np.abs(ls).sum(0)
    F[:, 10] = np.asarray(scene.opacity_logit, np.float32)
    F[:, 11:59] = np.asarray(scene.sh, np.float32).reshape(48, n).T
    return F, valid, E


def bf16_within(x, F, E):
    """Whether bf16 values x lie in [bf16(F - E), bf16(F + E)] (the bf16
    rounding of any value within E of F: the rounding is monotone)."""
    lo, hi = bf16(F - E), bf16(F + E)
    return (x >= lo) & (x <= hi)


def coverage_bound(scene, cam, region_xy, plain_sel, doubt_px=1e-3):
    """(coverage, lo, hi): rendered_coverage and the interval a float32
    implementation's label lies in: its two sums within
    oracle.weight_sums_bound (pixel-centre region tests within doubt_px of
    the boundary taken either way), the ratio and its float32 division; where
    the sum over all pixels may be 0, any value in [0, 1] (a splat that may
    reach no pixel takes its plain bit)."""
    sp = _o.preprocess(scene, cam)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    off, ids = _o.tile_lists(sp, _o.depth_order(sp), tx, ty)
    H, W = cam.height, cam.width
    py, px = np.mgrid[0:H, 0:W]
    pxf, pyf = px.ravel().astype(np.float64), py.ravel().astype(np.float64)
    xy = np.asarray(region_xy, np.float64).reshape(-1, 2)
    inside = point_in_polygon(pxf, pyf, xy).astype(np.float64)
    dist = np.full(len(pxf), np.inf)
    for i in range(len(xy)):
        ax, ay = xy[i - 1]
        bx, by = xy[i]
        ex, ey = bx - ax, by - ay
        tt = np.clip(((pxf - ax) * ex + (pyf - ay) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
        dist = np.minimum(dist, np.hypot(pxf - ax - tt * ex, pyf - ay - tt * ey))
    doubt = (dist <= doubt_px).astype(np.float64)
    num = _o.weight_sums(sp, off, ids, inside, 2)
    den = _o.weight_sums(sp, off, ids, np.ones(H * W), 2)
    bn = _o.weight_sums_bound(sp, off, ids, inside, 2, doubt=doubt)
    bd = _o.weight_sums_bound(sp, off, ids, np.ones(H * W), 2)
    plain = np.asarray(plain_sel, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        cov = np.where(den > 0, np.minimum(num / den, 1.0), plain)
        sure = den > bd
        lo = np.where(sure, np.maximum(num - bn, 0.0) / (den + bd) * (1 - 2.0 ** -22), 0.0)
        hi = np.where(sure, np.minimum((num + bn) / np.where(sure, den - bd, 1.0), 1.0)
                      * (1 + 2.0 ** -22), 1.0)
    hi = np.minimum(hi, 1.0)
    return cov, lo, hi


# ---------------------------------------------------------------------------
# network

def forward(theta, X, rnd=True):
    r = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    P = unpack(theta)
    x = r(X)
    z1 = x @ r(P["W1"]) + P["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ r(P["W2"]) + P["b2"]
    h2 = r(gelu(z2))
    o = h2 @ r(P["W3"]) + P["b3"]
    return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, o=o)


# A float32 implementation that rounds at the same points (bf16 features,
# weights and activations) differs from forward() only through (1) the
# accumulation of each product in float32, in any order (the error of a sum
# of m terms is at most gamma_m times the sum of their magnitudes, gamma_m =
# m u / (1 - m u); u = 2^-22 allows for additions that truncate), (2) its
# GELU approximation (GELU_ERR absolute plus a few float32 roundings) and (3)
# the bf16 rounding of each activation, which can go to the other neighbour
# when the value's uncertainty interval contains a rounding midpoint.
ACC_U = 2.0 ** -22
GELU_ERR = 4.1e-7
GELU_SLOPE = 1.13        # max |GELU'(z)| = 1.1289...


def _gamma(m):
    return m * ACC_U / (1.0 - m * ACC_U)


def _bf16_spread(v, d):
    """Largest distance between bf16(v) and the bf16 rounding of any value
    within d of v (0 where no rounding midpoint lies within d)."""
    h = bf16(v)
    d = d + 2.0 ** -24 * np.abs(v)       # the float32 step before the bf16 rounding
    return np.maximum(np.abs(bf16(v - d) - h), np.abs(bf16(v + d) - h))


def _forward_errors(theta, X):
    """forward() and, per element, bounds on the float32 implementation's
    departure from it: e1, e2, e3 for z1, z2, o; dh1, dh2 for the bf16
    activations h1, h2."""
    P = unpack(theta)
    f = forward(theta, X)
    W1, W2, W3 = bf16(P["W1"]), bf16(P["W2"]), bf16(P["W3"])
    g = _gamma(K + 1)
    e1 = g * (np.abs(f["x"]) @ np.abs(W1) + np.abs(P["b1"]))
    dh1 = _bf16_spread(gelu(f["z1"]), GELU_SLOPE * e1 + GELU_ERR + 4 * 2.0 ** -24 * np.abs(f["z1"]))
    e2 = dh1 @ np.abs(W2) + g * ((np.abs(f["h1"]) + dh1) @ np.abs(W2) + np.abs(P["b2"]))
    dh2 = _bf16_spread(gelu(f["z2"]), GELU_SLOPE * e2 + GELU_ERR + 4 * 2.0 ** -24 * np.abs(f["z2"]))
    e3 = dh2 @ np.abs(W3) + g * ((np.abs(f["h2"]) + dh2) @ np.abs(W3) + np.abs(P["b3"]))
    return f, dict(e1=e1, dh1=dh1, e2=e2, dh2=dh2, e3=e3)


def forward_bound(theta, X):
    """Per output element, a bound on |o - forward(theta, X)["o"]| for any
    float32 implementation that rounds at forward's points (see above).
    Returns (forward dict, bound [n, 4])."""
    f, e = _forward_errors(theta, X)
    return f, e["e3"]


def loss_grad(theta, X, sel, cov, rnd=True, batch=None):
    """Mean loss over the batch and its gradient (parameter-vector layout).
    batch: the batch size the sums are divided by (default len(X); larger
    when the batch also holds empty rows)."""
    r = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    P = unpack(theta)
    f = forward(theta, X, rnd)
    o = f["o"]
    B = len(X) if batch is None else batch
    y = np.asarray(sel, np.float64)
    cv = np.asarray(cov, np.float64)
    p0 = sigmoid(o[:, 0])
    pc = sigmoid(o[:, 1:4])
    bce = np.maximum(o[:, 0], 0) - y * o[:, 0] + np.log1p(np.exp(-np.abs(o[:, 0])))
    loss = float((bce + ((pc - cv[:, None]) ** 2).sum(1)).sum() / B)
    dz3 = np.zeros((len(X), N_OUT))
    dz3[:, 0] = (p0 - y) / B
    dz3[:, 1:] = 2.0 * (pc - cv[:, None]) * pc * (1 - pc) / B
    g = {}
    dz3r = r(dz3)
    g["W3"] = f["h2"].T @ dz3r
    g["b3"] = dz3.sum(0)
    dz2 = (dz3r @ r(P["W3"]).T) * gelu_grad(f["z2"])
    dz2r = r(dz2)
    g["W2"] = f["h1"].T @ dz2r
    g["b2"] = dz2.sum(0)
    dz1 = (dz2r @ r(P["W2"]).T) * gelu_grad(f["z1"])
    dz1r = r(dz1)
    g["W1"] = f["x"].T @ dz1r
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


# The backward of a float32 implementation that rounds at loss_grad's points
# departs from it through the forward's departures (above), float32 sigmoid
# and GELU' (SIG_ERR, GGRAD_ERR absolute: a few roundings of values below 1
# and 1.13), their slopes (|sigmoid'| <= 1/4, |d/dp 2 (p - c) p (1 - p)| <=
# 5/2 for p, c in [0, 1], |GELU''| <= 2 phi(0) < GELU_CURV), the float32
# sums over the rows (any order and grouping: at most ACC_DEPTH additions
# per term beyond the rows themselves, e.g. a block's 128 rows, its 8 warps
# and the blocks) and the bf16 rounding of dz3, dz2, dz1, which can go to
# the other neighbour like an activation's. A sum over the rows whose
# grouping puts at most `depth` additions between any row's term and the
# result (len(X) for plain sums in any order; e.g. 128 + blocks for sums of
# blocks of 128 rows) errs by at most gamma_depth times the sum of the
# magnitudes.
SIG_ERR = 2.0 ** -20
GGRAD_ERR = 2.0 ** -20
GELU_CURV = 0.8


def grad_bound(theta, X, sel, cov, batch=None, depth=None):
    """loss_grad(theta, X, sel, cov, batch=batch) and, per parameter, a bound
    on the float32 implementation's departure from its gradient; depth: the
    most additions on any row's path in the implementation's row sums
    (default len(X) + 8: any order).
    Returns (loss, grad, bound), grad and bound in the parameter layout."""
    P = unpack(theta)
    f, e = _forward_errors(theta, X)
    loss, grad = loss_grad(theta, X, sel, cov, batch=batch)
    B = len(X) if batch is None else batch
    W2r, W3r = bf16(P["W2"]), bf16(P["W3"])
    o = f["o"]
    y = np.asarray(sel, np.float64)
    cv = np.asarray(cov, np.float64)
    p = sigmoid(o)
    dp = 0.25 * e["e3"] + SIG_ERR
    dz3 = np.empty_like(o)
    dz3[:, 0] = (p[:, 0] - y) / B
    dz3[:, 1:] = 2.0 * (p[:, 1:] - cv[:, None]) * p[:, 1:] * (1 - p[:, 1:]) / B
    d3 = (np.concatenate([dp[:, :1], 2.5 * dp[:, 1:]], 1) + 2.0 ** -21) / B
    gr = _gamma(len(X) + 8 if depth is None else depth)

    def wgrad(A, dA, D, s):
        # |A^T D - A'^T D'| for |A - A'| <= dA, |D - D'| <= s, float32 sums
        aA, aD = np.abs(A), np.abs(D)
        return aA.T @ s + dA.T @ aD + dA.T @ s + gr * ((aA + dA).T @ (aD + s))

    def delta(Dr, s, Wr, z, ez):
        # dz = (Dr Wr^T) GELU'(z) with Dr within s, z within ez, float32 sums of H terms
        a = Dr @ Wr.T
        da = s @ np.abs(Wr).T + _gamma(Wr.shape[1] + 1) * ((np.abs(Dr) + s) @ np.abs(Wr).T)
        gg = gelu_grad(z)
        dgg = GELU_CURV * ez + GGRAD_ERR
        dz = a * gg
        return dz, da * (np.abs(gg) + dgg) + np.abs(a) * dgg + 2.0 ** -22 * np.abs(dz)

    b = {}
    s3 = _bf16_spread(dz3, d3)
    b["W3"] = wgrad(f["h2"], e["dh2"], bf16(dz3), s3)
    b["b3"] = d3.sum(0) + gr * np.abs(dz3).sum(0)
    dz2, d2 = delta(bf16(dz3), s3, W3r, f["z2"], e["e2"])
    s2 = _bf16_spread(dz2, d2)
    b["W2"] = wgrad(f["h1"], e["dh1"], bf16(dz2), s2)
    b["b2"] = d2.sum(0) + gr * np.abs(dz2).sum(0)
    dz1, d1 = delta(bf16(dz2), s2, W2r, f["z1"], e["e1"])
    s1 = _bf16_spread(dz1, d1)
    b["W1"] = wgrad(f["x"], np.zeros_like(f["x"]), bf16(dz1), s1)
    b["b1"] = d1.sum(0) + gr * np.abs(dz1).sum(0)
    return loss, grad, pack(b)


def decisions(o, plain_sel, valid, delta):
    """Selection and per-channel tint weights of the learned path with the
    plain fallback: outside the learned domain or where
    |sigmoid(o0) - 1/2| < delta, the plain bit (and the plain bit as a binary
    weight); elsewhere the network's bit and sigmoid(o1..3).
    Returns (sel, weights [n, 3], fallback mask)."""
    p = sigmoid(o[:, 0])
    fb = valid & (np.abs(p - 0.5) < delta)
    plain = np.asarray(plain_sel, np.float64)
    use_plain = ~valid | fb
    sel = np.where(use_plain, plain_sel, p > 0.5).astype(np.uint8)
    w = np.where(use_plain[:, None], plain[:, None], sigmoid(o[:, 1:4]))
    return sel, w, fb
