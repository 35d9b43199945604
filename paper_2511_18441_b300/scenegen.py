"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras, selection regions
and colour matrices.

This module only *draws inputs*. It holds none of the method's arithmetic (no
projection, no spherical-harmonic evaluation, no blending) and imports neither
the CUDA binding nor the CPU oracle, so both sides can consume the same arrays.

Scene layout (structure of arrays, float32 unless stated):
    xyz            (3, n)      world-space centres mu
    log_scale      (3, n)      per-axis log of the scale matrix S (Eq. 1)
    quat           (4, n)      rotation R as a quaternion, (w, x, y, z), unnormalised
    opacity_logit  (n,)        the opacity sigma of Eq. 3 before a sigmoid
    sh             (16, 3, n)  SH coefficients C_l^m of Eq. 2, index k = l*l + l + m,
                               one row per (k, colour channel)

Recipe (the paper evaluates on MipNeRF360 captures, which are not available;
these draws stand in for them): centres are uniform on sphere and square-plane
surfaces with counts proportional to area, plus isotropic N(0, 0.01) jitter;
log-scales N(-4.5, 0.5) per axis; rotations are normalised N(0, I4) draws
(uniform on SO(3)); opacity logits N(0, 1.5); one palette colour per surface
with N(0, 0.05) RGB noise on the DC term and N(0, 0.03) on higher orders.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PALETTE = np.array(
    [[0.85, 0.15, 0.15], [0.15, 0.75, 0.20], [0.20, 0.30, 0.85],
     [0.90, 0.80, 0.15], [0.15, 0.80, 0.80], [0.80, 0.20, 0.75]],
    dtype=np.float64)

# The DC basis function is the constant 1/(2 sqrt(pi)); a DC coefficient of
# (colour - 0.5) * 2 sqrt(pi) therefore shows roughly `colour` from any view.
_DC_FROM_COLOUR = 2.0 * math.sqrt(math.pi)


@dataclass
class Scene:
    xyz: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.xyz.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.xyz[:, idx]),
                     np.ascontiguousarray(self.log_scale[:, idx]),
                     np.ascontiguousarray(self.quat[:, idx]),
                     np.ascontiguousarray(self.opacity_logit[idx]),
                     np.ascontiguousarray(self.sh[:, :, idx]))

    def concat(self, other: "Scene") -> "Scene":
        return Scene(np.concatenate([self.xyz, other.xyz], 1),
                     np.concatenate([self.log_scale, other.log_scale], 1),
                     np.concatenate([self.quat, other.quat], 1),
                     np.concatenate([self.opacity_logit, other.opacity_logit]),
                     np.concatenate([self.sh, other.sh], 2))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.xyz, self.log_scale, self.quat,
                                      self.opacity_logit, self.sh))


@dataclass
class Camera:
    """Pinhole camera. Pixel (i, j) has its centre at continuous coordinates
    (i, j); view space is +x right, +y down, +z forward."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_view: np.ndarray            # (3, 4) float32, rows [R | t]
    cam_pos: np.ndarray                  # (3,) float32, world position
    z_near: float = 0.2


@dataclass
class Region:
    """Screen-space selection region in continuous pixel coordinates.
    kind 'box': xy = [[u0, v0], [u1, v1]], half-open [u0, u1) x [v0, v1).
    kind 'polygon': xy = (k, 2) vertices, even-odd rule."""
    kind: str
    xy: np.ndarray


@dataclass
class Edit:
    region: Region
    color_matrix: np.ndarray             # (3, 3) float32, row-major, acts on RGB
    select_camera: Camera | None = None  # None: the render camera


@dataclass
class Workload:
    name: str
    scene: Scene
    camera: Camera
    edit: Edit | None
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))


# ----------------------------------------------------------------------------
# surfaces

def _unit_vectors(rng, k):
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_rotation(rng):
    """Uniformly random orthonormal frame: QR of a Gaussian 3x3 matrix with
    the signs of R's diagonal folded into Q."""
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def make_scene(n: int, seed: int, half_extent: float, n_spheres: int,
               sphere_radius: tuple, n_planes: int = 0,
               plane_side: tuple = (2.0, 5.0)) -> Scene:
    """Draw n Gaussians on random spheres/planes inside [-h, h]^3.

    Draw order is frozen: surfaces, then per-surface counts, then points,
    jitter, log-scales, quaternions, opacity logits, DC noise, higher orders.
    """
    rng = np.random.default_rng(seed)
    h = half_extent
    # surfaces: (kind, centre, size, rotation)
    surfaces = []
    for _ in range(n_spheres):
        c = rng.uniform(-h, h, size=3)
        r = rng.uniform(*sphere_radius)
        surfaces.append(("sphere", c, r, None))
    for _ in range(n_planes):
        c = rng.uniform(-h, h, size=3)
        s = rng.uniform(*plane_side)
        surfaces.append(("plane", c, s, _random_rotation(rng)))
    area = np.array([4 * math.pi * s[2] ** 2 if s[0] == "sphere" else s[2] ** 2
                     for s in surfaces])
    counts = rng.multinomial(n, area / area.sum())
    xyz = np.empty((n, 3))
    colour = np.empty((n, 3))
    o = 0
    for si, (kind, c, size, rot) in enumerate(surfaces):
        k = int(counts[si])
        if k == 0:
            continue
        if kind == "sphere":
            p = c + size * _unit_vectors(rng, k)
        else:
            uv = rng.uniform(-0.5 * size, 0.5 * size, size=(k, 2))
            local = np.concatenate([uv, np.zeros((k, 1))], 1)
            p = c + local @ rot.T
        xyz[o:o + k] = p
        colour[o:o + k] = PALETTE[si % len(PALETTE)]
        o += k
    xyz += rng.normal(0.0, 0.01, size=(n, 3))
    log_scale = rng.normal(-4.5, 0.5, size=(n, 3))
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    opacity_logit = rng.normal(0.0, 1.5, size=n)
    dc = (colour + rng.normal(0.0, 0.05, size=(n, 3)) - 0.5) * _DC_FROM_COLOUR
    rest = rng.normal(0.0, 0.03, size=(15, 3, n))
    sh = np.empty((16, 3, n))
    sh[0] = dc.T
    sh[1:] = rest
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f32(xyz.T), f32(log_scale.T), f32(quat.T), f32(opacity_logit), f32(sh))


# ----------------------------------------------------------------------------
# cameras

def look_at_camera(width, height, fovy_deg, eye, target, up=(0.0, -1.0, 0.0),
                   z_near=0.2) -> Camera:
    """Camera at `eye` looking at `target`; `up` is the world direction that
    appears upwards on screen (view +y points down)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    right = np.cross(fwd, up)
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])               # rows: view axes in world
    t = -R @ eye
    fy = height / (2.0 * math.tan(math.radians(fovy_deg) / 2.0))
    w2v = np.concatenate([R, t[:, None]], 1).astype(np.float32)
    return Camera(width, height, float(fy), float(fy), (width - 1) / 2.0,
                  (height - 1) / 2.0, w2v, eye.astype(np.float32), z_near)


def axis_camera(width, height, fovy_deg, distance) -> Camera:
    """Camera at (0, 0, -distance) looking along +z with +y down: the view
    rotation is the identity."""
    return look_at_camera(width, height, fovy_deg, (0.0, 0.0, -distance), (0.0, 0.0, 0.0),
                          up=(0.0, -1.0, 0.0))


def ring_cameras(n_views, radius, resolutions, seed, fovy_deg=60.0):
    """n_views cameras on a ring of `radius` in the y = 0 plane looking at the
    origin, each with a resolution drawn uniformly from `resolutions`."""
    rng = np.random.default_rng(seed)
    cams = []
    for k in range(n_views):
        a = 2 * math.pi * k / n_views
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        eye = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        cams.append(look_at_camera(w, h, fovy_deg, eye, (0.0, 0.0, 0.0)))
    return cams


# ----------------------------------------------------------------------------
# regions and colour matrices

def box_region(u0, v0, u1, v1) -> Region:
    return Region("box", np.array([[u0, v0], [u1, v1]], np.float32))


def pixel_box_region(x0, y0, size_x, size_y) -> Region:
    """The box covering pixels [x0, x0+size_x) x [y0, y0+size_y): pixel
    centres are integers, so the continuous box starts half a pixel earlier."""
    return box_region(x0 - 0.5, y0 - 0.5, x0 + size_x - 0.5, y0 + size_y - 0.5)


def box_as_polygon(region: Region) -> Region:
    """A box region as the 4-vertex polygon with the same corners."""
    (u0, v0), (u1, v1) = np.asarray(region.xy, np.float32)
    return Region("polygon", np.array([[u0, v0], [u1, v0], [u1, v1], [u0, v1]], np.float32))


def shoelace_area(xy) -> float:
    x, y = np.asarray(xy, np.float64).T
    return 0.5 * abs(float(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1))))


def polygon_region(width, height, n_vertices, area_fraction, seed) -> Region:
    """Star-shaped polygon centred on the image: vertex k at angle
    2 pi k / n + U(-pi/(2n), pi/(2n)) and radius R * U(0.75, 1.25), with R
    scaled so that the polygon's area is area_fraction * W * H."""
    rng = np.random.default_rng(seed)
    ang = 2 * math.pi * np.arange(n_vertices) / n_vertices + rng.uniform(
        -math.pi / (2 * n_vertices), math.pi / (2 * n_vertices), size=n_vertices)
    rad = rng.uniform(0.75, 1.25, size=n_vertices)
    unit = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    R = math.sqrt(area_fraction * width * height / shoelace_area(unit))
    xy = unit * R + np.array([(width - 1) / 2.0, (height - 1) / 2.0])
    return Region("polygon", xy.astype(np.float32))


def tint_matrix(t) -> np.ndarray:
    """The per-channel tint t as a colour matrix diag(t)."""
    return np.diag(np.asarray(t, np.float64)).astype(np.float32)


def hue_rotation_matrix(deg) -> np.ndarray:
    """Rotation of RGB space by `deg` about the grey axis (1, 1, 1)/sqrt(3)
    (Rodrigues' formula); it maps grey to grey."""
    a = math.radians(deg)
    k = np.ones(3) / math.sqrt(3.0)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    M = np.eye(3) + math.sin(a) * K + (1 - math.cos(a)) * (K @ K)
    return M.astype(np.float32)


# ----------------------------------------------------------------------------
# named workloads

def tiny_workload(n=10_000, seed=0, width=256, height=256) -> Workload:
    """10k Gaussians on 4 spheres (radius 0.2-0.5) in the unit cube, a 256x256
    camera at distance 2.5 with a 60 degree vertical field of view, a centred
    64x64 pixel box and the tint (0.9, 0.4, 0.2)."""
    scene = make_scene(n, seed, 0.5, 4, (0.2, 0.5))
    cam = axis_camera(width, height, 60.0, 2.5)
    bx = (width - 64) // 2
    by = (height - 64) // 2
    edit = Edit(pixel_box_region(bx, by, 64, 64), tint_matrix((0.9, 0.4, 0.2)))
    return Workload("tiny", scene, cam, edit)


def paper_scale_workload(n=1_000_000, seed=1, width=1920, height=1080,
                         hue_deg=90.0, polygon_seed=None) -> Workload:
    """n Gaussians on 40 spheres (radius 2-5) and 20 square planes (side 2-5)
    in a 10x10x10 box, one 1920x1080 camera at distance 14 with a 60 degree
    vertical field of view, a 12-vertex polygon covering 15% of the image and
    a hue rotation."""
    scene = make_scene(n, seed, 5.0, 40, (2.0, 5.0), 20, (2.0, 5.0))
    cam = axis_camera(width, height, 60.0, 14.0)
    region = polygon_region(width, height, 12, 0.15,
                            seed if polygon_seed is None else polygon_seed)
    edit = Edit(region, hue_rotation_matrix(hue_deg))
    return Workload(f"paper_{n}", scene, cam, edit)


@dataclass
class BatchWorkload:
    name: str
    scenes: list                         # list of Scene
    views: list                          # list of (scene index, Camera, Edit)


BATCH_RESOLUTIONS = ((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def batched_workload(sizes=(500_000, 1_000_000, 2_000_000, 4_000_000), views_per_scene=16,
                     resolutions=BATCH_RESOLUTIONS, seed=3) -> BatchWorkload:
    """Several scenes of the paper-scale generator (different seeds), each
    seen by `views_per_scene` cameras on a ring of radius 14 around the
    origin with resolutions drawn uniformly from `resolutions`. Each scene has
    its own edit: a pixel box covering the central quarter of its first ring
    camera's image (the selection camera of all its views, so that every view
    shows the same selected Gaussians recoloured) and its own tint."""
    scenes, views = [], []
    for k, n in enumerate(sizes):
        scenes.append(make_scene(int(n), seed + 17 * k, 5.0, 40, (2.0, 5.0), 20, (2.0, 5.0)))
        cams = ring_cameras(views_per_scene, 14.0, resolutions, seed + 31 * k)
        c0 = cams[0]
        region = pixel_box_region(c0.width // 4, c0.height // 4, c0.width // 2, c0.height // 2)
        rng = np.random.default_rng(seed + 53 * k)
        edit = Edit(region, tint_matrix(rng.uniform(0.2, 1.0, 3)), select_camera=c0)
        for cam in cams:
            views.append((k, cam, edit))
    return BatchWorkload(f"batch_{len(sizes)}x{views_per_scene}", scenes, views)


def random_polygons(count, width, height, seed, n_vertices=12, area=(0.05, 0.25)):
    """`count` star-shaped polygons (as polygon_region) with area fractions
    drawn from U(area) and centres drawn uniformly from the middle 60% of the
    image."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        reg = polygon_region(width, height, n_vertices, float(rng.uniform(*area)),
                             int(rng.integers(1 << 31)))
        shift = np.array([rng.uniform(-0.3, 0.3) * width, rng.uniform(-0.3, 0.3) * height])
        out.append(Region("polygon", (reg.xy + shift).astype(np.float32)))
    return out


# parameter vector of the selection MLP 59 -> 64 -> 64 -> 4: W1 [64][64]
# (input-major, rows 59..63 zero: padding inputs), b1 [64], W2 [64][64],
# b2 [64], W3 [64][4], b3 [4]
MLP_SHAPES = ((64, 64), (64,), (64, 64), (64,), (64, 4), (4,))
MLP_FAN_IN = (59, 59, 64, 64, 64, 64)
MLP_PARAMS = 8580


def mlp_init(seed) -> np.ndarray:
    """Initial MLP parameters: every weight and bias U(-1/sqrt(fan_in),
    1/sqrt(fan_in)) of its layer (the common default for linear layers)."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape, fan in zip(MLP_SHAPES, MLP_FAN_IN):
        b = 1.0 / math.sqrt(fan)
        parts.append(rng.uniform(-b, b, size=shape).astype(np.float32).reshape(-1))
    theta = np.concatenate(parts)
    theta[59 * 64:64 * 64] = 0.0   # W1 rows of the padding inputs
    assert theta.size == MLP_PARAMS
    return theta


def to_half(sh: np.ndarray, kind: str) -> np.ndarray:
    """Round float32 SH to float16 ('f16') or bfloat16 ('bf16', round to
    nearest even); returns the 16-bit payload as uint16 for bf16 and float16
    for f16."""
    if kind == "f16":
        return sh.astype(np.float16)
    if kind == "bf16":
        u = np.ascontiguousarray(sh, np.float32).view(np.uint32).astype(np.uint64)
        rounding = ((u >> 16) & 1) + 0x7FFF
        return ((u + rounding) >> 16).astype(np.uint16)
    raise ValueError(kind)


def from_half(a: np.ndarray, kind: str) -> np.ndarray:
    """Exact float32 value of 16-bit SH payloads produced by to_half."""
    if kind == "f16":
        return a.astype(np.float32)
    if kind == "bf16":
        return (a.astype(np.uint32) << 16).view(np.float32)
    raise ValueError(kind)
