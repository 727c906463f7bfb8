"""Seeded synthetic inputs for the CT volume ray caster.

This module only *makes inputs*: scalar volumes, 256-entry RGBA transfer-function tables and
camera records. It contains no step of the rendering method (no resampling, classification,
compositing, brick tables or gradients), so both the CUDA path and the CPU oracle can consume
its arrays without sharing any of the method's arithmetic.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` and is deterministic for a
given seed and shape. Volumes are returned as C-ordered arrays of shape ``(nz, ny, nx)``
(x fastest), voxel (i, j, k) sitting at the point (x, y, z) = (i, j, k).

The paper's CT data (a DICOM series, Sec. "Results") and its figures are not available; the
recipes below stand in for them with the value ranges of CT in Hounsfield units (HU): air
-1000, soft tissue 0..80 HU with noise, contrast-filled vessels 300 HU, bone 700..1500 HU.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Hounsfield window used to index CT transfer functions (12-bit CT range).
CT_LO = -1024.0
CT_HI = 3071.0
# Window of the 12-bit phantom.
PHANTOM_LO = 0.0
PHANTOM_HI = 4095.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _paint_ellipsoid(vol, center, semi, rot, value, mode):
    """Set (mode='set') or add (mode='add') `value` inside a rotated ellipsoid (voxel centres)."""
    nz, ny, nx = vol.shape
    ext = float(max(semi))
    lo = [max(0, int(math.floor(c - ext)) - 1) for c in center]
    hi = [min(n, int(math.ceil(c + ext)) + 2) for c, n in zip(center, (nx, ny, nz))]
    if any(h <= l for l, h in zip(lo, hi)):
        return
    z, y, x = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                          np.arange(lo[0], hi[0]), indexing="ij")
    rel = np.stack([x - center[0], y - center[1], z - center[2]], axis=-1).astype(np.float64)
    loc = rel @ rot  # coordinates in the ellipsoid frame
    inside = ((loc / np.asarray(semi)) ** 2).sum(-1) <= 1.0
    sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    if mode == "add":
        sub[inside] += value
    else:
        sub[inside] = value


def _paint_capsule(vol, p0, p1, radius, value):
    """Set `value` at voxel centres within `radius` of the segment p0-p1. Works through the
    bounding box 16 z-planes at a time, each restricted to the part of the box that the
    segment's points within reach of those planes can touch (same per-voxel test)."""
    nz, ny, nx = vol.shape
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    lo = np.maximum(np.floor(np.minimum(p0, p1) - radius) - 1, 0).astype(int)
    hi = np.minimum(np.ceil(np.maximum(p0, p1) + radius) + 2, [nx, ny, nz]).astype(int)
    if np.any(hi <= lo):
        return
    seg = p1 - p0
    for za in range(lo[2], hi[2], 16):
        zb = min(int(hi[2]), za + 16)
        # a voxel in planes za .. zb-1 within radius of the segment has its closest segment
        # point at z in [za - radius, zb - 1 + radius]
        if abs(seg[2]) > 1e-12:
            ta = (za - radius - 1.0 - p0[2]) / seg[2]
            tb = (zb + radius + 1.0 - p0[2]) / seg[2]
            ta, tb = max(min(ta, tb), 0.0), min(max(ta, tb), 1.0)
            if ta > tb:
                continue
        else:
            if p0[2] < za - radius - 1.0 or p0[2] > zb + radius + 1.0:
                continue
            ta, tb = 0.0, 1.0
        q0, q1 = p0 + ta * seg, p0 + tb * seg
        xlo = max(int(math.floor(min(q0[0], q1[0]) - radius)) - 1, int(lo[0]))
        xhi = min(int(math.ceil(max(q0[0], q1[0]) + radius)) + 2, int(hi[0]))
        ylo = max(int(math.floor(min(q0[1], q1[1]) - radius)) - 1, int(lo[1]))
        yhi = min(int(math.ceil(max(q0[1], q1[1]) + radius)) + 2, int(hi[1]))
        if xhi <= xlo or yhi <= ylo:
            continue
        z, y, x = np.meshgrid(np.arange(za, zb), np.arange(ylo, yhi), np.arange(xlo, xhi),
                              indexing="ij")
        pts = np.stack([x, y, z], axis=-1).astype(np.float64)
        t = np.clip(((pts - p0) @ seg) / max(seg @ seg, 1e-12), 0.0, 1.0)
        dist2 = ((pts - (p0 + t[..., None] * seg)) ** 2).sum(-1)
        vol[za:zb, ylo:yhi, xlo:xhi][dist2 <= radius * radius] = value


def phantom(n: int = 64, seed: int = 1, n_ellipsoids: int = 10) -> np.ndarray:
    """Seeded 3D Shepp-Logan-style phantom: `n_ellipsoids` rotated ellipsoids with additive
    intensities, clamped to the 12-bit range [0, 4095]; returns uint16 of shape (n, n, n).

    The first ellipsoid is a large 'skull' shell of intensity 2000; the others are drawn
    with centres in the middle half of the cube, semi-axes in [0.08n, 0.3n] and additive
    intensities in [-600, 1500]. No canonical Shepp-Logan parameter table is used.
    """
    rng = _rng(seed)
    acc = np.zeros((n, n, n), np.float64)
    c = (n - 1) / 2.0
    _paint_ellipsoid(acc, (c, c, c), (0.46 * n, 0.40 * n, 0.43 * n), np.eye(3), 2000.0, "add")
    for _ in range(n_ellipsoids - 1):
        center = rng.uniform(0.25 * n, 0.75 * n, 3)
        semi = rng.uniform(0.08 * n, 0.30 * n, 3)
        rot = _random_rotation(rng)
        value = float(rng.uniform(-600.0, 1500.0))
        _paint_ellipsoid(acc, center, semi, rot, value, "add")
    return np.clip(np.rint(acc), 0, 4095).astype(np.uint16)


def _smooth_field(rng, shape, lo, hi, cell=64):
    """Trilinear upsampling of a coarse uniform random grid: a smooth field in [lo, hi].
    Returns a function of (z0, z1) giving planes z0 .. z1-1 (x and y are interpolated once on
    the coarse planes, z per request: the same sums as interpolating the whole volume)."""
    nz, ny, nx = shape
    coarse = rng.uniform(lo, hi, (nz // cell + 2, ny // cell + 2, nx // cell + 2))

    def axis_weights(n):
        t = np.arange(n, dtype=np.float64) / cell
        i0 = np.floor(t).astype(int)
        return i0, t - i0

    out = coarse
    for axis, n in ((2, nx), (1, ny)):
        i0, w = axis_weights(n)
        a = np.take(out, i0, axis=axis)
        b = np.take(out, i0 + 1, axis=axis)
        shp = [1, 1, 1]
        shp[axis] = n
        w = w.reshape(shp)
        out = a * (1.0 - w) + b * w
    iz, wz = axis_weights(nz)

    def planes(z0, z1):
        w = wz[z0:z1].reshape(-1, 1, 1)
        a = np.take(out, iz[z0:z1], axis=0)
        b = np.take(out, iz[z0:z1] + 1, axis=0)
        return a * (1.0 - w) + b * w
    return planes


def ct_volume(shape=(400, 512, 512), seed: int = 3, n_bones: int = 30,
              n_vessels: int = 40) -> np.ndarray:
    """Synthetic CT in Hounsfield units, int16 of shape (nz, ny, nx).

    * air -1000 outside an elliptic body cylinder along z (semi-axes about 0.42 nx, 0.33 ny);
    * soft tissue inside: a seeded smooth field in [0, 80] HU plus N(0, 10) noise, rounded;
    * `n_bones` rotated bone ellipsoids, constant 700..1500 HU, two semi-axes in 6..24 and
      one in 15..60 voxels (elongated like long bones; all scaled by nx/512);
    * `n_vessels` straight contrast-filled capsules at 300 HU, radius 2..6 voxels.
    Later writes win: vessels over bone over tissue. Generation runs slab by slab in z so
    that the noise draw does not depend on available memory.
    """
    nz, ny, nx = shape
    rng = _rng(seed)
    scale = nx / 512.0
    cx = (nx - 1) / 2.0 + rng.uniform(-0.02, 0.02) * nx
    cy = (ny - 1) / 2.0 + rng.uniform(-0.02, 0.02) * ny
    ax = 0.42 * nx * rng.uniform(0.95, 1.05)
    ay = 0.33 * ny * rng.uniform(0.95, 1.05)
    vol = np.full(shape, -1000, np.int16)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    body = ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0
    tissue = _smooth_field(rng, shape, 0.0, 80.0)
    slab = 32
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        noise = rng.standard_normal((z1 - z0, ny, nx)) * 10.0
        vals = np.rint(tissue(z0, z1) + noise).astype(np.int16)
        sl = vol[z0:z1]
        sl[:, body] = vals[:, body]

    def point_in_body():
        while True:
            x = rng.uniform(cx - ax, cx + ax)
            y = rng.uniform(cy - ay, cy + ay)
            if ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 <= 0.8:
                return x, y

    for _ in range(n_bones):
        x, y = point_in_body()
        z = rng.uniform(0.05 * nz, 0.95 * nz)
        semi = np.array([rng.uniform(6.0, 24.0), rng.uniform(6.0, 24.0),
                         rng.uniform(15.0, 60.0)]) * scale
        rot = _random_rotation(rng)
        value = int(rng.integers(700, 1501))
        _paint_ellipsoid(vol, (x, y, z), semi, rot, value, "set")
    for _ in range(n_vessels):
        x, y = point_in_body()
        z = rng.uniform(0.0, nz)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        length = rng.uniform(0.2, 0.6) * nz
        p0 = np.array([x, y, z])
        p1 = p0 + d * length
        radius = float(rng.uniform(2.0, 6.0))
        _paint_capsule(vol, p0, p1, radius, 300)
    return vol


def ct_float_downsampled(seed: int = 7, n: int = 512) -> np.ndarray:
    """float32 CT of shape (n/2,)*3: the int16 CT generator at n^3, 2x2x2 block mean."""
    v = ct_volume((n, n, n), seed=seed).astype(np.float32)
    h = n // 2
    return v.reshape(h, 2, h, 2, h, 2).mean(axis=(1, 3, 5), dtype=np.float64).astype(np.float32)


# ---------------------------------------------------------------------------------------
# Transfer-function tables (inputs): 256 x RGBA float32, entry k sits at index u = k.

def tf_from_control_points(xs, rgba) -> np.ndarray:
    """Piecewise-linear table through control points (xs in index units 0..255), extended
    constantly outside them."""
    xs = np.asarray(xs, np.float64)
    rgba = np.asarray(rgba, np.float64)
    k = np.arange(256, dtype=np.float64)
    return np.stack([np.interp(k, xs, rgba[:, c]) for c in range(4)], axis=1).astype(np.float32)


def tf_random(seed: int = 2, n_points: int = 4) -> np.ndarray:
    """`n_points` seeded control points: distinct sorted integer positions in [0, 255] and
    RGBA drawn uniformly in [0, 1]."""
    rng = _rng(seed)
    xs = np.sort(rng.choice(256, size=n_points, replace=False))
    rgba = rng.uniform(0.0, 1.0, (n_points, 4))
    return tf_from_control_points(xs, rgba)


_CT_POINTS = np.array([
    # HU,     r,    g,    b,    alpha (per unit voxel length)
    [-1024.0, 0.00, 0.00, 0.00, 0.00],
    [150.0, 0.70, 0.10, 0.08, 0.00],
    [300.0, 0.85, 0.12, 0.10, 0.06],
    [450.0, 0.90, 0.45, 0.30, 0.03],
    [700.0, 1.00, 0.92, 0.82, 0.35],
    [1500.0, 1.00, 0.98, 0.95, 0.80],
    [3071.0, 1.00, 1.00, 1.00, 0.90],
])


def tf_ct(seed: int | None = None, lo: float = CT_LO, hi: float = CT_HI) -> np.ndarray:
    """CT transfer function: transparent below 150 HU, a low-alpha red band around 300 HU
    (contrast-filled vessels) and white, high-alpha bone from 700 HU. With a seed, the
    control points are jittered (HU by +-30, colours and alphas by +-20%), giving the
    seeded family used for serving and for gradient targets."""
    pts = _CT_POINTS.copy()
    if seed is not None:
        rng = _rng(seed)
        pts[2:-1, 0] += rng.uniform(-30.0, 30.0, len(pts) - 3)
        pts[1:, 1:] = np.clip(pts[1:, 1:] * rng.uniform(0.8, 1.2, (len(pts) - 1, 4)), 0.0, 1.0)
        pts[1, 4] = 0.0
    xs = (pts[:, 0] - lo) / (hi - lo) * 255.0
    return tf_from_control_points(xs, pts[:, 1:])


_CT_DENSE_POINTS = np.array([
    # HU,     r,    g,    b,    alpha (per unit voxel length)
    [-1024.0, 0.00, 0.00, 0.00, 0.000],
    [-300.0, 0.55, 0.35, 0.30, 0.000],
    [-100.0, 0.75, 0.50, 0.42, 0.004],
    [40.0, 0.85, 0.55, 0.45, 0.012],
    [120.0, 0.90, 0.60, 0.50, 0.020],
    [300.0, 0.95, 0.20, 0.15, 0.080],
    [700.0, 1.00, 0.92, 0.82, 0.300],
    [3071.0, 1.00, 1.00, 1.00, 0.800],
])


def tf_ct_dense(lo: float = CT_LO, hi: float = CT_HI) -> np.ndarray:
    """Dense CT transfer function: air transparent, soft tissue (0-80 HU) semi-transparent at
    about 0.01-0.02 opacity per voxel, vessels and bone more opaque. Rays through the body run
    for hundreds of samples and nearly every occupied brick is resampled throughout -- the
    regime where the stencil's gather and FP32 work, not empty-space skipping, set the
    frame time."""
    xs = (_CT_DENSE_POINTS[:, 0] - lo) / (hi - lo) * 255.0
    return tf_from_control_points(xs, _CT_DENSE_POINTS[:, 1:])


# ---------------------------------------------------------------------------------------
# Cameras (inputs). Fields mirror the C struct used on both sides of the parity tests.

@dataclasses.dataclass
class Camera:
    ortho: int
    eye: tuple
    center: tuple
    up: tuple
    fovy_deg: float
    ortho_extent: tuple
    width: int
    height: int

    def as_float32(self) -> "Camera":
        f = lambda v: tuple(float(np.float32(x)) for x in v)  # noqa: E731
        return Camera(int(self.ortho), f(self.eye), f(self.center), f(self.up),
                      float(np.float32(self.fovy_deg)), f(self.ortho_extent),
                      int(self.width), int(self.height))


def ortho_z_camera(dims, width: int, height: int) -> Camera:
    """Orthographic view along +z covering the x-y extent of the volume box: pixel (i, j)
    maps to x = (i + 0.5) * nx / width - 0.5, y = (j + 0.5) * ny / height - 0.5 and the ray
    starts on the front face z = -0.5."""
    nx, ny, nz = dims
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    return Camera(1, (cx, cy, -0.5), (cx, cy, cz), (0.0, -1.0, 0.0), 0.0,
                  (float(nx), float(ny)), width, height).as_float32()


def orbit_camera(rng_or_seed, dims, width: int, height: int, fovy_deg: float = 30.0) -> Camera:
    """Perspective camera on a seeded orbit around the volume centre: azimuth uniform in
    [0, 2 pi), elevation uniform in [-30, 30] degrees, up = +y, distance R / sin(fovy / 2)
    with R the half-diagonal of the volume box, so the bounding sphere fills the view."""
    rng = _rng(rng_or_seed) if isinstance(rng_or_seed, (int, np.integer)) else rng_or_seed
    nx, ny, nz = dims
    c = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    radius = 0.5 * math.sqrt(nx * nx + ny * ny + nz * nz)
    dist = radius / math.sin(math.radians(fovy_deg) / 2.0)
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = math.radians(rng.uniform(-30.0, 30.0))
    eye = c + dist * np.array([math.cos(el) * math.sin(az), math.sin(el),
                               math.cos(el) * math.cos(az)])
    return Camera(0, tuple(eye), tuple(c), (0.0, 1.0, 0.0), fovy_deg, (0.0, 0.0),
                  width, height).as_float32()


def orbit_cameras(seed: int, k: int, dims, width: int, height: int,
                  fovy_deg: float = 30.0) -> list[Camera]:
    rng = _rng(seed)
    return [orbit_camera(rng, dims, width, height, fovy_deg) for _ in range(k)]


def dims_of(vol: np.ndarray):
    """(nx, ny, nz) of a (nz, ny, nx) array."""
    nz, ny, nx = vol.shape
    return nx, ny, nz
