"""FP64 CPU oracle for the CT volume ray caster -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (``paper_2005_01442_gb300``) never imports it, and the
two share no code: this wrapper loads ``liborc.so`` built from ``vrc_oracle.c`` with gcc.

Functions mirror the steps of the method (Sec. "Methodology" of the paper: ray casting with
cubic-spline resampling, post-classification, block decomposition with empty space leaping
and early ray termination). See ``vrc_oracle.c`` for the readings taken where the paper is
silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")

DTYPES = {np.dtype(np.uint16): 0, np.dtype(np.int16): 1, np.dtype(np.float32): 2}


class Camera(C.Structure):
    _fields_ = [("ortho", C.c_int), ("eye", C.c_float * 3), ("center", C.c_float * 3),
                ("up", C.c_float * 3), ("fovy_deg", C.c_float), ("ortho_extent", C.c_float * 2),
                ("width", C.c_int), ("height", C.c_int)]


class Params(C.Structure):
    _fields_ = [("step", C.c_double), ("ert", C.c_double), ("brick", C.c_int),
                ("interp", C.c_int), ("preclass", C.c_int), ("shade", C.c_int),
                ("preint", C.c_int), ("ka", C.c_double), ("kd", C.c_double), ("ks", C.c_double),
                ("shininess", C.c_double), ("open_alpha", C.c_int)]


class Ball(C.Structure):
    _fields_ = [("enabled", C.c_int), ("c", C.c_double * 3), ("r", C.c_double)]


def build(force: bool = False) -> str:
    """Compile liborc.so (gcc, -O2, OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.orc_bspline_weights.argtypes = [C.c_double, dp]
        L.orc_bspline_dweights.argtypes = [C.c_double, dp]
        L.orc_sample.argtypes = [vp, ip, ip, ip, ip, C.c_double, C.c_double, C.c_double]
        L.orc_sample.restype = C.c_double
        L.orc_sample_linear.argtypes = [vp, ip, ip, ip, ip, C.c_double, C.c_double, C.c_double]
        L.orc_sample_linear.restype = C.c_double
        L.orc_sample_rgba.argtypes = [vp, ip, ip, ip, ip, C.c_double, C.c_double, C.c_double,
                                      ip, ip, vp, C.c_double, C.c_double, dp]
        L.orc_gradient.argtypes = [vp, ip, ip, ip, ip, C.c_double, C.c_double, C.c_double, dp]
        L.orc_preint_table.argtypes = [vp, C.c_double, vp]
        L.orc_preint_table.restype = ip
        L.orc_classify.argtypes = [C.c_double, vp, C.c_double, C.c_double, dp]
        L.orc_ray.argtypes = [C.POINTER(Camera), vp, ip, ip, dp, dp, dp, dp]
        L.orc_ray.restype = C.c_int
        L.orc_bricks.argtypes = [vp, ip, ip, ip, ip, ip, vp, vp]
        L.orc_occupancy.argtypes = [vp, vp, ip, C.c_long, vp, C.c_float, C.c_float, vp]
        L.orc_cellmask.argtypes = [vp, ip, ip, ip, ip, vp, C.c_float, C.c_float, vp]
        L.orc_brick_aabbs.argtypes = [vp, ip, ip, ip, ip, vp, vp]
        L.orc_render.argtypes = [vp, ip, ip, ip, ip, vp, C.c_double, C.c_double,
                                 C.POINTER(Camera), C.POINTER(Params), vp, C.POINTER(Ball), vp,
                                 C.c_long, vp, vp, vp, vp]
        L.orc_render_grad.argtypes = [vp, ip, ip, ip, ip, vp, C.c_double, C.c_double,
                                      C.POINTER(Camera), C.POINTER(Params), vp, vp, C.c_long,
                                      vp, vp, vp]
        L.orc_set_threads.argtypes = [ip]
        L.orc_get_threads.restype = ip
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _cam(cam) -> Camera:
    c = Camera()
    c.ortho = int(cam.ortho)
    c.eye[:] = [float(x) for x in cam.eye]
    c.center[:] = [float(x) for x in cam.center]
    c.up[:] = [float(x) for x in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.ortho_extent[:] = [float(x) for x in cam.ortho_extent]
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def bspline_weights(f: float) -> np.ndarray:
    w = (C.c_double * 4)()
    lib().orc_bspline_weights(float(f), w)
    return np.array(w[:])


def bspline_dweights(f: float) -> np.ndarray:
    w = (C.c_double * 4)()
    lib().orc_bspline_dweights(float(f), w)
    return np.array(w[:])


def sample(vol: np.ndarray, p) -> float:
    """Cubic B-spline value of `vol` (nz, ny, nx) at the point p = (x, y, z)."""
    vol = np.ascontiguousarray(vol)
    nz, ny, nx = vol.shape
    return float(lib().orc_sample(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, *map(float, p)))


def sample_linear(vol: np.ndarray, p) -> float:
    """Trilinear value of `vol` (nz, ny, nx) at the point p = (x, y, z)."""
    vol = np.ascontiguousarray(vol)
    nz, ny, nx = vol.shape
    return float(lib().orc_sample_linear(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz,
                                         *map(float, p)))


def sample_rgba(vol: np.ndarray, p, tf: np.ndarray, lo: float, hi: float, interp: int = 0,
                preclass: int = 0) -> np.ndarray:
    """rgba of the sample at p under an interpolation (0 cubic, 1 trilinear) and
    classification (0 post, 1 pre) variant."""
    vol = np.ascontiguousarray(vol)
    tf = np.ascontiguousarray(tf, np.float32)
    nz, ny, nx = vol.shape
    out = (C.c_double * 4)()
    lib().orc_sample_rgba(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, *map(float, p), int(interp),
                          int(preclass), _ptr(tf), float(lo), float(hi), out)
    return np.array(out[:])


def preint_table(tf: np.ndarray, step: float) -> np.ndarray:
    """(256, 256, 4) pre-integration table (front entry, back entry; associated rgb,
    opacity) for slabs of length `step`."""
    tf = np.ascontiguousarray(tf, np.float32)
    out = np.empty((256, 256, 4), np.float64)
    if lib().orc_preint_table(_ptr(tf), float(step), _ptr(out)) != 0:
        raise ValueError("orc_preint_table failed")
    return out


def gradient(vol: np.ndarray, p) -> np.ndarray:
    """Gradient of the cubic B-spline field of `vol` (nz, ny, nx) at p = (x, y, z)."""
    vol = np.ascontiguousarray(vol)
    nz, ny, nx = vol.shape
    out = (C.c_double * 3)()
    lib().orc_gradient(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, *map(float, p), out)
    return np.array(out[:])


def classify(s: float, tf: np.ndarray, lo: float, hi: float) -> np.ndarray:
    tf = np.ascontiguousarray(tf, np.float32)
    out = (C.c_double * 4)()
    lib().orc_classify(float(s), _ptr(tf), float(lo), float(hi), out)
    return np.array(out[:])


def ray(cam, dims, px: int, py: int):
    """(origin, direction, t_in, t_out, hit) of the ray through pixel (px, py)."""
    o = (C.c_double * 3)()
    d = (C.c_double * 3)()
    t0 = C.c_double()
    t1 = C.c_double()
    dm = np.asarray(dims, np.int32)
    hit = lib().orc_ray(C.byref(_cam(cam)), _ptr(dm), int(px), int(py), o, d, C.byref(t0),
                        C.byref(t1))
    return np.array(o[:]), np.array(d[:]), t0.value, t1.value, bool(hit)


def bricks(vol: np.ndarray, B: int):
    """Per-brick (min, max) over the apron box, arrays of shape (nbz, nby, nbx)."""
    vol = np.ascontiguousarray(vol)
    nz, ny, nx = vol.shape
    nb = tuple((n + B - 1) // B for n in (nz, ny, nx))
    mn = np.empty(nb, vol.dtype)
    mx = np.empty(nb, vol.dtype)
    rc = lib().orc_bricks(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, int(B), _ptr(mn), _ptr(mx))
    if rc != 0:
        raise ValueError(f"orc_bricks failed ({rc})")
    return mn, mx


def occupancy(mn: np.ndarray, mx: np.ndarray, tf: np.ndarray, lo: float, hi: float) -> np.ndarray:
    mn = np.ascontiguousarray(mn)
    mx = np.ascontiguousarray(mx)
    tf = np.ascontiguousarray(tf, np.float32)
    occ = np.empty(mn.shape, np.uint8)
    rc = lib().orc_occupancy(_ptr(mn), _ptr(mx), DTYPES[mn.dtype], mn.size, _ptr(tf),
                             float(lo), float(hi), _ptr(occ))
    if rc != 0:
        raise ValueError(f"orc_occupancy failed ({rc})")
    return occ


def cellmask(vol: np.ndarray, tf: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Cell transparency bytes, shape (nz+1, ny+1, nx+1): entry [c2+1, c1+1, c0+1] is 0 when
    every sample with floor(p) = (c0, c1, c2) has alpha == 0 (see orc_cellmask)."""
    vol = np.ascontiguousarray(vol)
    tf = np.ascontiguousarray(tf, np.float32)
    nz, ny, nx = vol.shape
    out = np.empty((nz + 1, ny + 1, nx + 1), np.uint8)
    rc = lib().orc_cellmask(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, _ptr(tf), float(lo),
                            float(hi), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_cellmask failed ({rc})")
    return out


def _pix(pixels):
    if pixels is None:
        return None, 0
    p = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    return p, p.shape[0]


def render(vol, tf, lo, hi, cam, step, ert=1.0, brick=0, pixels=None, ball=None,
           return_margin=False, return_counts=False, return_executed=False, interp=0,
           preclass=0, phong=None, preint=0, occ=None):
    """FP64 render. Returns float64 (H, W, 4) (or (npix, 4) for a pixel list), plus the ERT
    margins, the (nominal, executed) sample counts and the per-pixel executed samples when
    asked. interp / preclass select the variant; phong = (ka, kd, ks, shininess) turns on
    headlight Blinn-Phong shading (cubic post-classification); preint 1 composites slabs
    between consecutive samples through the pre-integrated table (no skipping). occ replaces
    the brick occupancy of `brick` (a piece render passes the occupancy of its piece)."""
    vol = np.ascontiguousarray(vol)
    tf = np.ascontiguousarray(tf, np.float32)
    nz, ny, nx = vol.shape
    if brick and occ is None:
        mn, mx = bricks(vol, brick)
        occ = occupancy(mn, mx, tf, lo, hi)
    if occ is not None:
        occ = np.ascontiguousarray(occ, np.uint8)
    pix, npix = _pix(pixels)
    n = npix if pix is not None else cam.width * cam.height
    out = np.zeros((n, 4), np.float64)
    margin = np.empty(n, np.float64) if return_margin else None
    counts = np.zeros(2, np.int64)
    expp = np.zeros(n, np.int32) if return_executed else None
    sh = phong is not None
    ka, kd, ks, shin = phong if sh else (0.0, 0.0, 0.0, 1.0)
    par = Params(float(step), float(ert), int(brick), int(interp), int(preclass), int(sh),
                 int(preint), float(ka), float(kd), float(ks), float(shin))
    b = None
    if ball is not None:
        b = Ball(1, (C.c_double * 3)(*map(float, ball[0])), float(ball[1]))
    rc = lib().orc_render(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, _ptr(tf), float(lo),
                          float(hi), C.byref(_cam(cam)), C.byref(par), _ptr(occ),
                          C.byref(b) if b is not None else None, _ptr(pix), npix, _ptr(out),
                          _ptr(margin), _ptr(counts), _ptr(expp))
    if rc != 0:
        raise ValueError(f"orc_render failed ({rc})")
    img = out if pix is not None else out.reshape(cam.height, cam.width, 4)
    res = [img]
    if return_margin:
        res.append(margin if pix is not None else margin.reshape(cam.height, cam.width))
    if return_counts:
        res.append((int(counts[0]), int(counts[1])))
    if return_executed:
        res.append(expp if pix is not None else expp.reshape(cam.height, cam.width))
    return res[0] if len(res) == 1 else tuple(res)


def render_grad(vol, tf, lo, hi, cam, step, g, ert=1.0, brick=0, pixels=None, want_vol=True,
                open_alpha=False):
    """Reverse-mode gradient of sum(g * image) w.r.t. the TF (256, 4) and the voxels
    (vol.shape), in float64. open_alpha: at table opacity 0 take the opacity correction's
    derivative from above instead of from the clamped side (brick must be 0)."""
    vol = np.ascontiguousarray(vol)
    tf = np.ascontiguousarray(tf, np.float32)
    nz, ny, nx = vol.shape
    occ = None
    if brick:
        mn, mx = bricks(vol, brick)
        occ = occupancy(mn, mx, tf, lo, hi)
    pix, npix = _pix(pixels)
    g = np.ascontiguousarray(np.asarray(g, np.float64).reshape(-1, 4))
    gtf = np.zeros((256, 4), np.float64)
    gvol = np.zeros(vol.shape, np.float64) if want_vol else None
    par = Params(float(step), float(ert), int(brick), 0, 0, 0, 0, 0.0, 0.0, 0.0, 1.0,
                 int(bool(open_alpha)))
    rc = lib().orc_render_grad(_ptr(vol), DTYPES[vol.dtype], nx, ny, nz, _ptr(tf), float(lo),
                               float(hi), C.byref(_cam(cam)), C.byref(par), _ptr(occ),
                               _ptr(pix), npix, _ptr(g), _ptr(gtf), _ptr(gvol))
    if rc != 0:
        raise ValueError(f"orc_render_grad failed ({rc})")
    return gtf, gvol


# ------------------------------------------------------------------------------------------
# Object-order rendering with sort-last compositing (see "pieces" in vrc_oracle.c)


def brick_aabbs(vol: np.ndarray, tf: np.ndarray, lo: float, hi: float, B: int) -> np.ndarray:
    """Tight visible box of every brick, int16 (nbz, nby, nbx, 6): (lo_x, lo_y, lo_z, hi_x,
    hi_y, hi_z), half-open in cell coordinates (cell c holds the points with floor(p) = c);
    zeros for a brick with no open cell or an empty brick (see orc_brick_aabbs)."""
    vol = np.ascontiguousarray(vol)
    tf = np.ascontiguousarray(tf, np.float32)
    nz, ny, nx = vol.shape
    cm = cellmask(vol, tf, lo, hi)
    mn, mx = bricks(vol, B)
    occ = occupancy(mn, mx, tf, lo, hi)
    out = np.empty(occ.shape + (6,), np.int16)
    rc = lib().orc_brick_aabbs(_ptr(cm), nx, ny, nz, int(B), _ptr(occ), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_brick_aabbs failed ({rc})")
    return out


def piece_grid(dims, B: int, grid):
    """Pieces of a (gx, gy, gz) grid over the bricks of a volume of size dims = (nx, ny, nz):
    a list, piece index (sz * gy + sy) * gx + sx, of brick boxes (lo, hi), half-open, piece s
    of g along an axis holding bricks [floor(s nb / g), floor((s + 1) nb / g))."""
    nb = [(int(n) + B - 1) // B for n in dims]
    out = []
    for sz in range(grid[2]):
        for sy in range(grid[1]):
            for sx in range(grid[0]):
                s = (sx, sy, sz)
                out.append((tuple(s[k] * nb[k] // grid[k] for k in range(3)),
                            tuple((s[k] + 1) * nb[k] // grid[k] for k in range(3))))
    return out


def piece_cells(dims, B: int, blo, bhi):
    """Cell range [lo, hi) per axis of the bricks [blo, bhi): brick b holds the cells
    [bB, bB + B), brick 0 also cell -1, the last brick the cells up to n - 1."""
    nb = [(int(n) + B - 1) // B for n in dims]
    lo = tuple(-1 if blo[k] == 0 else blo[k] * B for k in range(3))
    hi = tuple(int(dims[k]) if bhi[k] == nb[k] else bhi[k] * B for k in range(3))
    return lo, hi


def piece_occupancy(occ: np.ndarray, blo, bhi) -> np.ndarray:
    """The brick occupancy (nbz, nby, nbx) with every brick outside [blo, bhi) set to 0."""
    m = np.zeros_like(occ)
    m[blo[2]:bhi[2], blo[1]:bhi[1], blo[0]:bhi[0]] = occ[blo[2]:bhi[2], blo[1]:bhi[1],
                                                         blo[0]:bhi[0]]
    return m


def render_piece(vol, tf, lo, hi, cam, step, brick, blo, bhi, ert=1.0, pixels=None, **kw):
    """Partial image (C, 1 - T) of the piece of bricks [blo, bhi): the samples whose brick lies
    in the piece, composited from T = 1 with their own early termination. Further keywords
    (the variant, return_margin) go to render()."""
    mn, mx = bricks(vol, brick)
    occ = piece_occupancy(occupancy(mn, mx, tf, lo, hi), blo, bhi)
    return render(vol, tf, lo, hi, cam, step, ert=ert, brick=brick, pixels=pixels, occ=occ,
                  **kw)


def pixel_piece_order(cam, dims, cell_boxes, pixels) -> np.ndarray:
    """Per pixel, the piece indices in the order in which its ray enters the pieces' boxes
    (point sets floor(p) in [lo, hi), clipped to the volume box [-0.5, n - 0.5]), pieces the
    ray does not meet last in index order. int (npix, K)."""
    pix, npix = _pix(pixels)
    K = len(cell_boxes)
    order = np.empty((npix, K), np.int64)
    for i in range(npix):
        o, d, t_in, t_out, hit = ray(cam, dims, int(pix[i, 0]), int(pix[i, 1]))
        ent = []
        for k, (clo, chi) in enumerate(cell_boxes):
            t0, t1 = t_in, t_out
            for a in range(3):
                lo_a = max(float(clo[a]), -0.5)
                hi_a = min(float(chi[a]), float(dims[a]) - 0.5)
                if d[a] != 0.0:
                    ta, tb = (lo_a - o[a]) / d[a], (hi_a - o[a]) / d[a]
                    t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
                elif not (lo_a <= o[a] < hi_a):
                    t0, t1 = 1.0, 0.0
            ent.append((0, t0, k) if (hit and t0 < t1) else (1, 0.0, k))
        order[i] = [k for _, _, k in sorted(ent)]
    return order


def composite(partials: np.ndarray, order: np.ndarray) -> np.ndarray:
    """Over-composition of partial images (K, npix, 4) per pixel in the given order (npix, K):
    C += T C_k, T *= 1 - A_k from C = 0, T = 1; returns (C, 1 - T), float64 (npix, 4)."""
    partials = np.asarray(partials, np.float64)
    K, npix, _ = partials.shape
    out = np.zeros((npix, 4), np.float64)
    for i in range(npix):
        C = np.zeros(3)
        T = 1.0
        for k in order[i]:
            C += T * partials[k, i, :3]
            T *= 1.0 - partials[k, i, 3]
        out[i, :3] = C
        out[i, 3] = 1.0 - T
    return out
