"""FP64 CPU oracle (ctypes front end of ``recogs_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``. The product package never imports
it, and it imports nothing from the product package: inputs arrive as plain
numpy arrays or duck-typed scene/camera/edit objects with the fields that the
seeded generator produces.

Method: ReCoGS (arXiv 2511.18441), Eq. 1-3 of Sec. 3.1, the tint c* = t.c and
the SH-only edit of Sec. 3.3, HWC output of Sec. 4.2. Pins live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recogs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

f64p = C.POINTER(C.c_double)
f32p = C.POINTER(C.c_float)
u8p = C.POINTER(C.c_uint8)
i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "recogs_oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", _LIB, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("view", C.c_double * 12),
                ("cam_pos", C.c_double * 3), ("z_near", C.c_double)]


class Edit(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_vertices", C.c_int), ("xy", f64p), ("M", C.c_double * 9),
                ("select_cam", Camera)]


class Margins(C.Structure):
    _fields_ = [("eps_pos", C.c_double), ("eps_rel", C.c_double), ("eps_k", C.c_double),
                ("eps_pix", C.c_double), ("eps_cov", C.c_double), ("eps_exp", C.c_double),
                ("eps_depth", C.c_double), ("impact", C.c_double)]


class Splats(C.Structure):
    _fields_ = [("u", f64p), ("v", f64p), ("depth", f64p), ("cov2d", f64p), ("conic", f64p),
                ("opacity", f64p), ("rgb", f64p), ("extent", f64p), ("rect", i32p),
                ("valid", u8p), ("visible", u8p), ("selected", u8p), ("sel_flag", u8p),
                ("fp_flag", u8p), ("alt_rgb", f64p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.oracle_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, f64p]
        L.oracle_quat_to_rotation.argtypes = [f64p, f64p]
        L.oracle_covariance3d.argtypes = [f64p, f64p, f64p]
        L.oracle_select.argtypes = [C.c_int64, f32p, C.POINTER(Edit), C.c_double, u8p, u8p]
        L.oracle_recolor.argtypes = [C.c_int64, f32p, u8p, f64p, f64p]
        L.oracle_preprocess.argtypes = [C.c_int64, f32p, f32p, f32p, f32p, f32p, C.POINTER(Camera),
                                        C.POINTER(Edit), C.POINTER(Margins), C.POINTER(Splats),
                                        C.c_int]
        L.oracle_preprocess.restype = C.c_int
        L.oracle_depth_order.argtypes = [C.c_int64, C.POINTER(Splats), i64p]
        L.oracle_depth_order.restype = C.c_int64
        L.oracle_render_pixels.argtypes = [C.POINTER(Splats), i64p, C.c_int64, C.c_int64, i32p, i32p,
                                           f64p, C.POINTER(Margins), f64p, f64p, u8p, i32p, C.c_int]
        L.oracle_tile_lists.argtypes = [C.POINTER(Splats), i64p, C.c_int64, C.c_int, C.c_int, i64p,
                                        i32p]
        L.oracle_tile_lists.restype = C.c_int64
        L.oracle_render_tiles.argtypes = [C.POINTER(Splats), i64p, i32p, C.c_int, C.c_int, C.c_int64,
                                          i32p, f64p, C.POINTER(Margins), f64p, f64p, u8p, i32p,
                                          C.c_int]
        L.oracle_render_tiles_depth.argtypes = [C.POINTER(Splats), i64p, i32p, C.c_int, C.c_int,
                                                C.c_int64, i32p, f64p, C.POINTER(Margins), f64p,
                                                f64p, u8p, i32p, C.c_double, f64p, u8p, C.c_int]
        L.oracle_color_grad_tiles.argtypes = [C.POINTER(Splats), i64p, i32p, C.c_int, C.c_int,
                                              f64p, f64p]
        L.oracle_color_grad_bound_tiles.argtypes = [C.c_int64, C.POINTER(Splats), i64p, i32p,
                                                    C.c_int, C.c_int, f64p, C.POINTER(Margins),
                                                    f64p]
        L.oracle_weight_sums_bound_tiles.argtypes = [C.c_int64, C.POINTER(Splats), i64p, i32p,
                                                     C.c_int, C.c_int, f64p, f64p, C.c_int,
                                                     C.POINTER(Margins), f64p]
        L.oracle_sh_grad.argtypes = [C.c_int64, f32p, C.POINTER(Camera), f64p, f64p, f64p]
        L.oracle_pixel_outcomes.argtypes = [C.POINTER(Splats), i64p, i32p, C.c_int, C.c_int, i64p,
                                            C.c_int64, C.c_int64, i32p, i32p, f64p,
                                            C.POINTER(Margins), C.c_double, C.c_int64, f64p, i64p,
                                            C.c_int]
        L.oracle_weight_sums_tiles.argtypes = [C.POINTER(Splats), i64p, i32p, C.c_int, C.c_int,
                                               f64p, C.c_int, f64p]
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# structs

def camera_struct(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    v = np.asarray(cam.world_to_view, np.float64).reshape(12)
    for k in range(12):
        c.view[k] = float(v[k])
    for k in range(3):
        c.cam_pos[k] = float(np.asarray(cam.cam_pos, np.float64)[k])
    c.z_near = float(cam.z_near)
    return c


def edit_struct(edit, cam):
    """Returns (Edit, keep-alive list)."""
    e = Edit()
    if edit is None:
        e.kind = 0
        return e, []
    xy = np.ascontiguousarray(np.asarray(edit.region.xy, np.float64).reshape(-1))
    e.kind = 1 if edit.region.kind == "box" else 2
    e.n_vertices = len(xy) // 2
    e.xy = _ptr(xy, f64p)
    M = np.asarray(edit.color_matrix, np.float64).reshape(9)
    for k in range(9):
        e.M[k] = float(M[k])
    e.select_cam = camera_struct(edit.select_camera if edit.select_camera is not None else cam)
    return e, [xy]


def margins(cam, eps_pos=None, eps_rel=1e-5, eps_k=1e-6, eps_pix=2e-5, eps_cov=1e-5,
            eps_exp=4e-6, eps_depth=1e-12, impact=5e-5) -> Margins:
    """Decision margins: how far float32 arithmetic may move each quantity.

    eps_pos (selection and tile-range decisions) defaults to 1e-6 * max(W, H)
    px, the selection-boundary width read relative to the image size. The
    pixel-level margins bound a float32 implementation that keeps the
    pixel-to-centre offset to ~1e-6 px, covariance entries to ~1e-6 of their
    scale and the exponent to a few ulp; each default is 2.5-10x that bound.
    eps_depth: a depth within this distance (relative) of the midpoint
    between two float32 values may get either as its float32 key (a float32
    implementation carries the depth to ~1e-13 before rounding it). Two
    contributors whose keys may be equal may be blended in either order, so
    the pixel's colour is not unique there; such pixels are flagged.
    """
    m = Margins()
    m.eps_pos = float(1e-6 * max(cam.width, cam.height) if eps_pos is None else eps_pos)
    m.eps_rel = float(eps_rel)
    m.eps_k = float(eps_k)
    m.eps_pix = float(eps_pix)
    m.eps_cov = float(eps_cov)
    m.eps_exp = float(eps_exp)
    m.eps_depth = float(eps_depth)
    m.impact = float(impact)
    return m


# ---------------------------------------------------------------------------
# small pieces used by the pins

def sh_basis(x, y, z) -> np.ndarray:
    Y = np.zeros(16)
    lib().oracle_sh_basis(float(x), float(y), float(z), _ptr(Y, f64p))
    return Y


def quat_to_rotation(q) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().oracle_quat_to_rotation(_ptr(q, f64p), _ptr(R, f64p))
    return R.reshape(3, 3)


def covariance3d(q, log_scale) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    s = np.ascontiguousarray(log_scale, np.float64)
    S = np.zeros(9)
    lib().oracle_covariance3d(_ptr(q, f64p), _ptr(s, f64p), _ptr(S, f64p))
    return S.reshape(3, 3)


# ---------------------------------------------------------------------------
# pipeline pieces

def select(scene, edit, cam, eps_pos=None):
    """Selection bits and near-boundary flags of every splat centre."""
    n = scene.xyz.shape[1]
    xyz = np.ascontiguousarray(scene.xyz, np.float32)
    e, keep = edit_struct(edit, cam)
    scam = edit.select_camera if edit.select_camera is not None else cam
    eps = 1e-6 * max(scam.width, scam.height) if eps_pos is None else eps_pos
    sel = np.zeros(n, np.uint8)
    flag = np.zeros(n, np.uint8)
    lib().oracle_select(n, _ptr(xyz, f32p), C.byref(e), float(eps), _ptr(sel, u8p), _ptr(flag, u8p))
    return sel, flag


def recolor(sh, selected, M) -> np.ndarray:
    """FP64 recoloured SH coefficients, layout [16][3][n]."""
    sh = np.ascontiguousarray(sh, np.float32)
    n = sh.shape[-1]
    sel = np.ascontiguousarray(selected, np.uint8)
    Mm = np.ascontiguousarray(np.asarray(M, np.float64).reshape(9))
    out = np.zeros((16, 3, n))
    lib().oracle_recolor(n, _ptr(sh, f32p), _ptr(sel, u8p), _ptr(Mm, f64p), _ptr(out, f64p))
    return out


class SplatResult(dict):
    """Per-splat arrays from oracle_preprocess plus the ctypes view of them."""

    def struct(self) -> Splats:
        s = Splats()
        for name, t in (("u", f64p), ("v", f64p), ("depth", f64p), ("cov2d", f64p),
                        ("conic", f64p), ("opacity", f64p), ("rgb", f64p), ("extent", f64p),
                        ("rect", i32p), ("valid", u8p), ("visible", u8p), ("selected", u8p),
                        ("sel_flag", u8p), ("fp_flag", u8p), ("alt_rgb", f64p)):
            setattr(s, name, _ptr(self[name], t))
        return s


def preprocess(scene, cam, edit=None, mg=None, sh=None, threads=None) -> SplatResult:
    """Per-splat selection, recolour, projection, footprint and colour.
    `sh` overrides scene.sh (float32 [16][3][n], e.g. dequantised 16-bit)."""
    n = scene.xyz.shape[1]
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    xyz, ls, q, op = f32(scene.xyz), f32(scene.log_scale), f32(scene.quat), f32(scene.opacity_logit)
    shv = f32(scene.sh if sh is None else sh)
    r = SplatResult(
        u=np.zeros(n), v=np.zeros(n), depth=np.zeros(n), cov2d=np.zeros(3 * n),
        conic=np.zeros(3 * n), opacity=np.zeros(n), rgb=np.zeros(3 * n), extent=np.zeros(2 * n),
        rect=np.zeros(4 * n, np.int32), valid=np.zeros(n, np.uint8), visible=np.zeros(n, np.uint8),
        selected=np.zeros(n, np.uint8), sel_flag=np.zeros(n, np.uint8),
        fp_flag=np.zeros(n, np.uint8), alt_rgb=np.zeros(3 * n))
    camc = camera_struct(cam)
    e, keep = edit_struct(edit, cam)
    m = mg if mg is not None else margins(cam)
    s = r.struct()
    rc = lib().oracle_preprocess(n, _ptr(xyz, f32p), _ptr(ls, f32p), _ptr(q, f32p), _ptr(op, f32p),
                                 _ptr(shv, f32p), C.byref(camc), C.byref(e) if edit else None,
                                 C.byref(m), C.byref(s), _threads(threads))
    if rc != 0:
        raise RuntimeError("oracle_preprocess failed")
    r["n"] = n
    r["camera"] = cam
    r["margins"] = m
    return r


def depth_order(splats: SplatResult) -> np.ndarray:
    n = splats["n"]
    order = np.zeros(max(n, 1), np.int64)
    s = splats.struct()
    m = lib().oracle_depth_order(n, C.byref(s), _ptr(order, i64p))
    return order[:m].copy()


def render_pixels(splats: SplatResult, order, px, py, bg=(0.0, 0.0, 0.0), mg=None, threads=None):
    """Definitional render of pixels (px[j], py[j]): each walks every splat."""
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    order = np.ascontiguousarray(order, np.int64)
    npix = len(px)
    bgv = np.ascontiguousarray(bg, np.float64)
    rgb = np.zeros((npix, 3))
    T = np.zeros(npix)
    flag = np.zeros(npix, np.uint8)
    nc = np.zeros(npix, np.int32)
    m = mg if mg is not None else splats["margins"]
    s = splats.struct()
    lib().oracle_render_pixels(C.byref(s), _ptr(order, i64p), len(order), npix, _ptr(px, i32p),
                               _ptr(py, i32p), _ptr(bgv, f64p), C.byref(m), _ptr(rgb, f64p),
                               _ptr(T, f64p), _ptr(flag, u8p), _ptr(nc, i32p), _threads(threads))
    return dict(rgb=rgb, T=T, flag=flag, ncontrib=nc)


def tile_lists(splats: SplatResult, order, tiles_x, tiles_y):
    """(offsets[tiles+1], ids[P]) of per-tile (depth, index)-sorted lists."""
    order = np.ascontiguousarray(order, np.int64)
    s = splats.struct()
    offsets = np.zeros(tiles_x * tiles_y + 1, np.int64)
    P = lib().oracle_tile_lists(C.byref(s), _ptr(order, i64p), len(order), tiles_x, tiles_y,
                                _ptr(offsets, i64p), None)
    ids = np.zeros(max(P, 1), np.int32)
    lib().oracle_tile_lists(C.byref(s), _ptr(order, i64p), len(order), tiles_x, tiles_y,
                            _ptr(offsets, i64p), _ptr(ids, i32p))
    return offsets, ids[:P]


def depth_keys(splats: SplatResult):
    """Float32 depth keys: the float32 nearest each FP64 view depth, and a
    mask of the depths within eps_depth (relative) of a float32 rounding
    midpoint, whose key float32 arithmetic may round either way. A float32
    sort by (key, index) is the (depth, index) order of Eq. 3 except inside
    runs of equal keys."""
    d = np.asarray(splats["depth"], np.float64)
    eps = splats["margins"].eps_depth
    k = d.astype(np.float32)
    other = np.where(k.astype(np.float64) <= d, np.nextafter(k, np.float32(np.inf)),
                     np.nextafter(k, np.float32(-np.inf)))
    mid = 0.5 * (k.astype(np.float64) + other.astype(np.float64))
    amb = np.abs(d - mid) <= eps * np.abs(d)
    return k, amb


def pixel_outcomes(splats: SplatResult, offsets, ids, px, py, bg=(0.0, 0.0, 0.0), mg=None,
                   max_out=256, threads=None, tau=None):
    """Every outcome (r, g, b, T) of the binned render at pixels (px[j],
    py[j]) that the doubtful decisions allow (the oracle's flags): returns
    (outcomes [npix, max_out, 4], counts [npix]; -1 where there are more
    than max_out). With tau, each outcome also carries its median depth
    (outcomes [npix, max_out, 5]), the crossing of tau in doubt branching
    too."""
    cam = splats["camera"]
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    npix = len(px)
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    extra = np.ascontiguousarray(np.flatnonzero(splats["fp_flag"] > 0), np.int64)
    n_extra = len(extra)
    if n_extra == 0:
        extra = np.zeros(1, np.int64)
    bgv = np.ascontiguousarray(bg, np.float64)
    out = np.zeros((max(npix, 1), max_out, 5))
    cnt = np.zeros(max(npix, 1), np.int64)
    m = mg if mg is not None else splats["margins"]
    s = splats.struct()
    lib().oracle_pixel_outcomes(C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p), cam.width,
                                cam.height, _ptr(extra, i64p), n_extra, npix, _ptr(px, i32p),
                                _ptr(py, i32p), _ptr(bgv, f64p), C.byref(m),
                                float(tau) if tau is not None else 0.0, int(max_out),
                                _ptr(out, f64p), _ptr(cnt, i64p), _threads(threads))
    return (out[:npix] if tau is not None else out[:npix, :, :4]), cnt[:npix]


def render_tiles(splats: SplatResult, offsets, ids, tiles=None, bg=(0.0, 0.0, 0.0), mg=None,
                 threads=None, tau=None):
    """Binned render of the listed tiles (all by default) into full-size HWC
    arrays; pixels of other tiles are left at zero. With tau, also the median
    depth (Sec. 3.2.2) and its decision flags."""
    cam = splats["camera"]
    W, H = cam.width, cam.height
    tx = (W + 15) // 16
    ty = (H + 15) // 16
    if tiles is None:
        tiles = np.arange(tx * ty, dtype=np.int32)
    tiles = np.ascontiguousarray(tiles, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    bgv = np.ascontiguousarray(bg, np.float64)
    rgb = np.zeros((H, W, 3))
    T = np.zeros((H, W))
    flag = np.zeros((H, W), np.uint8)
    nc = np.zeros((H, W), np.int32)
    m = mg if mg is not None else splats["margins"]
    s = splats.struct()
    if tau is None:
        lib().oracle_render_tiles(C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p), W, H,
                                  len(tiles), _ptr(tiles, i32p), _ptr(bgv, f64p), C.byref(m),
                                  _ptr(rgb, f64p), _ptr(T, f64p), _ptr(flag, u8p), _ptr(nc, i32p),
                                  _threads(threads))
        return dict(rgb=rgb, T=T, flag=flag, ncontrib=nc)
    depth = np.zeros((H, W))
    dflag = np.zeros((H, W), np.uint8)
    lib().oracle_render_tiles_depth(C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p), W, H,
                                    len(tiles), _ptr(tiles, i32p), _ptr(bgv, f64p), C.byref(m),
                                    _ptr(rgb, f64p), _ptr(T, f64p), _ptr(flag, u8p),
                                    _ptr(nc, i32p), float(tau), _ptr(depth, f64p),
                                    _ptr(dflag, u8p), _threads(threads))
    return dict(rgb=rgb, T=T, flag=flag, ncontrib=nc, depth=depth, dflag=dflag)


# ---------------------------------------------------------------------------
# the SH-only refit (Sec. 3.3; Eq. 6 with lambda = 0, Eq. 7 restricted to the
# SH coefficients)

def l1_loss_grad(y, target):
    """L1 loss mean |y - target| over the N = H*W*3 values and its gradient
    sign(y - target) / N (Eq. 6 with the SSIM weight lambda = 0)."""
    y = np.asarray(y, np.float64)
    d = y - np.asarray(target, np.float64)
    N = d.size
    return float(np.abs(d).sum() / N), np.sign(d) / N


def color_grad(splats: SplatResult, offsets, ids, dLdy) -> np.ndarray:
    """dL/dc_i (shape [n, 3]) of the binned render for the image gradient
    dLdy (HWC); splats that do not contribute get 0."""
    cam = splats["camera"]
    n = splats["n"]
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    g = np.ascontiguousarray(dLdy, np.float64).reshape(-1)
    out = np.zeros(3 * max(n, 1))
    s = splats.struct()
    lib().oracle_color_grad_tiles(C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p), cam.width,
                                  cam.height, _ptr(g, f64p), _ptr(out, f64p))
    return out[:3 * n].reshape(n, 3)


def color_grad_bound(splats: SplatResult, offsets, ids, dLdy, mg=None) -> np.ndarray:
    """Per splat and channel ([n, 3]), a bound on how far the colour gradient
    of a float32 blend may lie from color_grad: float32 alpha and T within
    the margins of the render's error model, decisions in doubt (alpha
    against 1/255, the stop, validity, key ties) taken either way, and
    float32 sums over the pixels in any order."""
    cam = splats["camera"]
    n = splats["n"]
    mg = margins(cam) if mg is None else mg
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    g = np.ascontiguousarray(dLdy, np.float64).reshape(-1)
    out = np.zeros(3 * max(n, 1))
    s = splats.struct()
    lib().oracle_color_grad_bound_tiles(n, C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p),
                                        cam.width, cam.height, _ptr(g, f64p), C.byref(mg),
                                        _ptr(out, f64p))
    return out[:3 * n].reshape(n, 3)


def weight_sums_bound(splats: SplatResult, offsets, ids, pixel_weight, power, doubt=None,
                      mg=None) -> np.ndarray:
    """Per splat ([n]), a bound on how far a float32 blend's sums of
    weight_sums may lie from the oracle's (the error model of
    color_grad_bound); doubt ([H*W], optional): the largest change of each
    pixel's weight on the float32 side."""
    cam = splats["camera"]
    n = splats["n"]
    mg = margins(cam) if mg is None else mg
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    w = np.ascontiguousarray(pixel_weight, np.float64).reshape(-1)
    d = None if doubt is None else np.ascontiguousarray(doubt, np.float64).reshape(-1)
    out = np.zeros(max(n, 1))
    s = splats.struct()
    lib().oracle_weight_sums_bound_tiles(n, C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p),
                                         cam.width, cam.height, _ptr(w, f64p),
                                         _ptr(d, f64p) if d is not None else None, int(power),
                                         C.byref(mg), _ptr(out, f64p))
    return out[:n]


def weight_sums(splats: SplatResult, offsets, ids, pixel_weight, power) -> np.ndarray:
    """Per splat: sum_p pixel_weight[p] (alpha T)^power over its contributions."""
    cam = splats["camera"]
    n = splats["n"]
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    if len(ids) == 0:
        ids = np.zeros(1, np.int32)
    g = np.ascontiguousarray(pixel_weight, np.float64).reshape(-1)
    out = np.zeros(max(n, 1))
    s = splats.struct()
    lib().oracle_weight_sums_tiles(C.byref(s), _ptr(offsets, i64p), _ptr(ids, i32p), cam.width,
                                   cam.height, _ptr(g, f64p), int(power), _ptr(out, f64p))
    return out[:n]


def sh_grad(scene, splats: SplatResult, grad_rgb) -> np.ndarray:
    """dL/dC (layout [16][3][n]) from the colour gradient (Eq. 2)."""
    n = splats["n"]
    xyz = np.ascontiguousarray(scene.xyz, np.float32)
    g = np.ascontiguousarray(grad_rgb, np.float64).reshape(-1)
    out = np.zeros((16, 3, n))
    camc = camera_struct(splats["camera"])
    lib().oracle_sh_grad(n, _ptr(xyz, f32p), C.byref(camc), _ptr(splats["rgb"], f64p),
                         _ptr(g, f64p), _ptr(out, f64p))
    return out


# float32 evaluation of the SH basis at the normalised view direction: within
# SH_BASIS_ERR of Y_k (absolute; |Y_k| <= 3 for degree 3, a few roundings of
# the direction and of the polynomial)
SH_BASIS_ERR = 4e-6


def sh_grad_bound(scene, splats: SplatResult, grad_rgb, bound_rgb) -> np.ndarray:
    """[16][3][n]: a bound on how far a float32 SH gradient Y_k(d) [c > 0]
    g_c, fed a colour gradient within bound_rgb of grad_rgb, may lie from
    sh_grad(scene, splats, grad_rgb). The clamp c = max(f + 0.5, 0) may be
    decided either way where the float32 f + 0.5 may have the other sign
    (|f + 0.5| <= 2e-6 (1 + sum_k |C_k Y_k|))."""
    n = splats["n"]
    xyz = np.ascontiguousarray(scene.xyz, np.float32)
    ones = np.ones(3 * max(n, 1))
    Y = np.zeros((16, 3, max(n, 1)))
    camc = camera_struct(splats["camera"])
    lib().oracle_sh_grad(n, _ptr(xyz, f32p), C.byref(camc), _ptr(ones, f64p), _ptr(ones, f64p),
                         _ptr(Y, f64p))
    Y = Y[:, 0, :n]                                       # [16][n]
    sh = np.asarray(scene.sh, np.float64)[:, :, :n]       # [16][3][n]
    terms = sh * Y[:, None, :]
    f = terms.sum(0) + 0.5                                # [3][n]
    ef = 2e-6 * (1.0 + np.abs(terms).sum(0))
    g = np.asarray(grad_rgb, np.float64).reshape(n, 3).T  # [3][n]
    b = np.asarray(bound_rgb, np.float64).reshape(n, 3).T
    aY = np.abs(Y)[:, None, :] + SH_BASIS_ERR
    passed = aY * b + SH_BASIS_ERR * np.abs(g) + 2.0 ** -23 * np.abs(Y)[:, None, :] * (np.abs(g) + b)
    either = aY * (np.abs(g) + b)
    out = np.where(f > ef, passed, np.where(f < -ef, 0.0, either))
    return np.broadcast_to(out, (16, 3, n)).copy()


def adam_step(C, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (Kingma and Ba, 2015) with bias correction at step t
    (1-based); returns the new (C, m, v). The optimiser of the refit is not
    named by the paper; Adam is the optimiser of the 3DGS rasteriser it uses."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return C - lr * mh / (np.sqrt(vh) + eps), m, v


def render_image(scene, cam, edit=None, bg=(0.0, 0.0, 0.0), mg=None, sh=None, threads=None):
    """Full binned FP64 render; returns (image dict, splats, order, offsets, ids)."""
    sp = preprocess(scene, cam, edit, mg, sh=sh, threads=threads)
    order = depth_order(sp)
    tx = (cam.width + 15) // 16
    ty = (cam.height + 15) // 16
    offsets, ids = tile_lists(sp, order, tx, ty)
    img = render_tiles(sp, offsets, ids, None, bg, mg, threads)
    return img, sp, order, offsets, ids
