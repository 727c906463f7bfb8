"""Brute-force NumPy FP64 ray caster for tiny inputs -- test infrastructure only.

An independent second statement of the same reading as ``vrc_oracle.c``, written differently
on purpose so that the two can pin each other:

* the resampled value is the full kernel sum  s(p) = sum_m beta3(p - m) Vext[m]  over every
  grid point m of the volume extended by edge replication, with beta3 the centred cubic
  B-spline written piecewise (2/3 - t^2 + |t|^3/2 on |t| < 1, (2 - |t|)^3 / 6 on 1 <= |t| < 2);
* the camera is a matrix (right, up, forward) applied to screen offsets;
* the ray-box range uses a vectorised slab test;
* compositing runs over the midpoints of the step partition of [t_in, t_out].

Only usable for volumes of a few thousand voxels and images of a few dozen pixels.
"""
from __future__ import annotations

import math

import numpy as np

PAD = 3


def beta3(t):
    t = np.abs(np.asarray(t, np.float64))
    out = np.zeros_like(t)
    a = t < 1.0
    b = (t >= 1.0) & (t < 2.0)
    out[a] = 2.0 / 3.0 - t[a] ** 2 + 0.5 * t[a] ** 3
    out[b] = (2.0 - t[b]) ** 3 / 6.0
    return out


def dbeta3(t):
    """Derivative of beta3 (odd): -2t + 3t|t|/2 on |t| < 1, -sign(t)(2 - |t|)^2 / 2 on
    1 <= |t| < 2."""
    t = np.asarray(t, np.float64)
    a = np.abs(t)
    out = np.zeros_like(t)
    m1 = a < 1.0
    m2 = (a >= 1.0) & (a < 2.0)
    out[m1] = -2.0 * t[m1] + 1.5 * t[m1] * a[m1]
    out[m2] = -np.sign(t[m2]) * (2.0 - a[m2]) ** 2 / 2.0
    return out


def tent(t):
    """Linear B-spline (the trilinear kernel per axis): max(0, 1 - |t|)."""
    return np.maximum(0.0, 1.0 - np.abs(np.asarray(t, np.float64)))


class Field:
    """Volume extended by edge replication; s(p) by the full kernel sum with the cubic
    B-spline (kernel="cubic") or the tent (kernel="linear"). With `channels` (an array of
    shape vol.shape + (c,)), the same sum of those per-voxel values instead."""

    def __init__(self, vol, kernel="cubic", channels=None):
        v = np.asarray(vol if channels is None else channels, np.float64)
        if channels is None:
            v = v[..., None]
        self.ext = np.pad(v, [(PAD, PAD)] * 3 + [(0, 0)], mode="edge")
        nz, ny, nx = v.shape[:3]
        self.kern = beta3 if kernel == "cubic" else tent
        self.scalar = channels is None
        self.gx = np.arange(-PAD, nx + PAD, dtype=np.float64)
        self.gy = np.arange(-PAD, ny + PAD, dtype=np.float64)
        self.gz = np.arange(-PAD, nz + PAD, dtype=np.float64)

    def gradient(self, p):
        """Gradient of the cubic field at p (the kernel sum with one factor differentiated)."""
        bx, by, bz = beta3(p[0] - self.gx), beta3(p[1] - self.gy), beta3(p[2] - self.gz)
        dx, dy, dz = dbeta3(p[0] - self.gx), dbeta3(p[1] - self.gy), dbeta3(p[2] - self.gz)
        e = self.ext[..., 0]
        return np.array([np.einsum("k,j,i,kji->", bz, by, dx, e),
                         np.einsum("k,j,i,kji->", bz, dy, bx, e),
                         np.einsum("k,j,i,kji->", dz, by, bx, e)])

    def __call__(self, p):
        bx = self.kern(p[0] - self.gx)
        by = self.kern(p[1] - self.gy)
        bz = self.kern(p[2] - self.gz)
        r = np.einsum("k,j,i,kjic->c", bz, by, bx, self.ext)
        return float(r[0]) if self.scalar else r


def camera_rays(cam, dims):
    """Per-pixel (origin, unit direction) arrays of shape (H, W, 3)."""
    eye = np.asarray(cam.eye, np.float64)
    fwd = np.asarray(cam.center, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(cam.up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    M = np.stack([right, upv, fwd], axis=1)  # columns
    W, H = cam.width, cam.height
    ix = (np.arange(W) + 0.5) / W * 2.0 - 1.0
    iy = 1.0 - (np.arange(H) + 0.5) / H * 2.0
    sx, sy = np.meshgrid(ix, iy)  # (H, W)
    if cam.ortho:
        off = np.stack([sx * cam.ortho_extent[0] / 2, sy * cam.ortho_extent[1] / 2,
                        np.zeros_like(sx)], -1)
        org = eye + off @ M.T
        dirs = np.broadcast_to(fwd, org.shape).copy()
    else:
        th = math.tan(math.radians(cam.fovy_deg) / 2)
        scr = np.stack([sx * th * W / H, sy * th, np.ones_like(sx)], -1)
        dirs = scr @ M.T
        dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
        org = np.broadcast_to(eye, dirs.shape).copy()
    return org, dirs


def box_range(org, d, dims):
    lo = -0.5 * np.ones(3)
    hi = np.asarray(dims, np.float64) - 0.5
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo - org) / d
        tb = (hi - org) / d
    tmin = np.where(d != 0, np.minimum(ta, tb), np.where((org >= lo) & (org <= hi), -np.inf, np.inf))
    tmax = np.where(d != 0, np.maximum(ta, tb), np.where((org >= lo) & (org <= hi), np.inf, -np.inf))
    return max(0.0, tmin.max()), tmax.min()


def tf_lookup(s, tf, lo, hi):
    u = min(max((s - lo) / (hi - lo) * 255.0, 0.0), 255.0)
    k = np.arange(256, dtype=np.float64)
    return np.array([np.interp(u, k, tf[:, c].astype(np.float64)) for c in range(4)])


def preint_table(tf, ds, k=32):
    """(256, 256, 4) table: the k-sub-step composite of the table along the linear ramp of
    the index from the row entry to the column entry over the length ds (vectorised)."""
    tf = np.asarray(tf, np.float64)
    i = np.arange(256, dtype=np.float64)[:, None]
    j = np.arange(256, dtype=np.float64)[None, :]
    col = np.zeros((256, 256, 3))
    trans = np.ones((256, 256))
    amax = 1.0 - 2.0 ** -24
    for n in range(k):
        u = i + (j - i) * (n + 0.5) / k
        i0 = np.minimum(np.floor(u).astype(int), 254)
        f = u - i0
        rgba = (1.0 - f)[..., None] * tf[i0] + f[..., None] * tf[i0 + 1]
        alpha = 1.0 - (1.0 - np.clip(rgba[..., 3], 0.0, amax)) ** (ds / k)
        col += trans[..., None] * alpha[..., None] * rgba[..., :3]
        trans *= 1.0 - alpha
    return np.concatenate([col, (1.0 - trans)[..., None]], -1)


def render(vol, tf, lo, hi, cam, step, ert=1.0, interp=0, preclass=0, phong=None, preint=0,
           keep=None):
    """(H, W, 4) float64 image: front-to-back compositing over segment midpoints.
    interp 0/1: cubic B-spline / trilinear kernel; preclass 1: classify every voxel, then
    interpolate the rgba; phong (ka, kd, ks, shininess): headlight shading by the gradient of
    the cubic field, softened by eps = 0.01 (hi - lo); preint: slabs between consecutive
    samples through the pre-integration table, looked up bilinearly. keep(p) -> bool, when
    given, drops every sample point it rejects (a partial image of part of the volume)."""
    nz, ny, nx = vol.shape
    dims = (nx, ny, nz)
    kernel = "cubic" if interp == 0 else "linear"
    if preclass:
        rgba_vol = np.stack([tf_lookup(float(v), tf, lo, hi)
                             for v in np.asarray(vol, np.float64).ravel()])
        pre = Field(vol, kernel, rgba_vol.reshape(vol.shape + (4,)))
        sample = pre
    else:
        field = Field(vol, kernel)
        sample = lambda p: tf_lookup(field(p), tf, lo, hi)  # noqa: E731
    org, dirs = camera_rays(cam, dims)
    preint_tab = preint_table(tf, step) if preint else None
    img = np.zeros((cam.height, cam.width, 4))
    amax = 1.0 - 2.0 ** -24
    for j in range(cam.height):
        for i in range(cam.width):
            o, d = org[j, i], dirs[j, i]
            t0, t1 = box_range(o, d, dims)
            if not t1 > t0:
                continue
            edges = np.append(np.arange(t0, t1, step), t1)
            if edges.size > 1 and edges[-2] >= t1:
                edges = edges[:-1]
            col = np.zeros(3)
            trans = 1.0
            if preint:
                tab = preint_tab
                prev = None
                for a, b in zip(edges[:-1], edges[1:]):
                    p = o + 0.5 * (a + b) * d
                    u = min(max((field(p) - lo) / (hi - lo) * 255.0, 0.0), 255.0)
                    mid = 0.5 * (a + b)
                    if prev is not None:
                        u0, m0 = prev
                        i0, k0 = min(int(math.floor(u0)), 254), min(int(math.floor(u)), 254)
                        fi, fk = u0 - i0, u - k0
                        e = ((1 - fi) * ((1 - fk) * tab[i0, k0] + fk * tab[i0, k0 + 1])
                             + fi * ((1 - fk) * tab[i0 + 1, k0] + fk * tab[i0 + 1, k0 + 1]))
                        alpha = e[3]
                        length = mid - m0
                        if abs(length - step) > 1e-12 and alpha > 0.0:
                            a2 = 1.0 - (1.0 - alpha) ** (length / step)
                            e = e * (a2 / alpha)
                            alpha = a2
                        col += trans * e[:3]
                        trans *= 1.0 - alpha
                        if ert < 1.0 and 1.0 - trans > ert:
                            break
                    prev = (u, mid)
                img[j, i, :3] = col
                img[j, i, 3] = 1.0 - trans
                continue
            for a, b in zip(edges[:-1], edges[1:]):
                p = o + 0.5 * (a + b) * d
                if keep is not None and not keep(p):
                    continue
                rgba = sample(p)
                if phong is not None:
                    ka, kd, ks, shin = phong
                    g = field.gradient(p)
                    eps = 0.01 * (hi - lo)
                    nl = abs(float(g @ d)) / math.sqrt(float(g @ g) + eps * eps)
                    rgba = rgba.copy()
                    rgba[:3] = rgba[:3] * (ka + kd * nl) + ks * nl ** shin
                alpha = 1.0 - (1.0 - min(max(rgba[3], 0.0), amax)) ** (b - a)
                col += trans * alpha * rgba[:3]
                trans *= 1.0 - alpha
                if ert < 1.0 and 1.0 - trans > ert:
                    break
            img[j, i, :3] = col
            img[j, i, 3] = 1.0 - trans
    return img
