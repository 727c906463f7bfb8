"""Host logic of object-order rendering that needs no GPU: the visibility order of a piece grid
(vrc_grid_order) and the pixel rectangle of a box (vrc_box_rect), checked against the
geometry of each pixel's ray as the oracle casts it (slab tests along the ray)."""
import os
import shutil

import numpy as np
import pytest

from paper_2005_01442_gb300 import build, native, synth


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libvrc")
        build.build()
    return native.load()


def _cams(dims, w=36, h=28):
    nx, ny, nz = dims
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2)
    cams = list(synth.orbit_cameras(7, 5, dims, w, h))
    cams.append(synth.ortho_z_camera(dims, w, h))
    # oblique orthographic view from a corner
    cams.append(synth.Camera(1, (-40.0, -30.0, -50.0), c, (0.0, 1.0, 0.0), 0.0,
                             (120.0, 100.0), w, h).as_float32())
    # eye inside the volume, between cut planes, wide field of view
    cams.append(synth.Camera(0, (0.3 * nx, 0.6 * ny, 0.45 * nz), (nx, 0.2 * ny, nz),
                             (0.0, 1.0, 0.0), 100.0, (0.0, 0.0), w, h).as_float32())
    return cams


def _interval(o, d, t0, t1, lo, hi):
    for a in range(3):
        if d[a] != 0.0:
            ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
        elif not (lo[a] <= o[a] < hi[a]):
            return None
    return (t0, t1) if t1 > t0 + 1e-9 else None


@pytest.mark.parametrize("grid", [(2, 2, 2), (3, 1, 2), (1, 4, 1), (3, 3, 3)])
def test_grid_order_agrees_with_every_rays_entry_order(lib, orc, grid):
    # For every pixel, the pieces its ray crosses (positive length inside the volume) appear
    # in the global order in the order the ray enters them.
    dims, B = (64, 48, 40), 8
    pieces = orc.piece_grid(dims, B, grid)
    boxes = [orc.piece_cells(dims, B, blo, bhi) for blo, bhi in pieces]
    cuts = []
    for a in range(3):
        starts = sorted({clo[a] for clo, _ in boxes})
        cuts += [float(c) for c in starts[1:]]
    crossed_pairs = 0
    for cam in _cams(dims):
        order = native.grid_order(cam, grid, cuts)
        assert sorted(order) == list(range(len(pieces)))
        rank = {k: i for i, k in enumerate(order)}
        for py in range(0, cam.height, 3):
            for px in range(0, cam.width, 3):
                o, d, t0, t1, hit = orc.ray(cam, dims, px, py)
                if not hit:
                    continue
                met = []
                for k, (clo, chi) in enumerate(boxes):
                    lo = [max(float(clo[a]), -0.5) for a in range(3)]
                    hi = [min(float(chi[a]), dims[a] - 0.5) for a in range(3)]
                    iv = _interval(o, d, t0, t1, lo, hi)
                    if iv is not None:
                        met.append((iv[0], k))
                met.sort()
                ranks = [rank[k] for _, k in met]
                assert ranks == sorted(ranks), (cam, px, py, met)
                crossed_pairs += max(len(met) - 1, 0)
    assert crossed_pairs > 100


def test_grid_order_rejects_bad_cuts(lib):
    cam = synth.orbit_cameras(1, 1, (32, 32, 32), 8, 8)[0]
    with pytest.raises(native.VrcError):
        native.grid_order(cam, (3, 1, 1), [20.0, 10.0])  # not increasing
    with pytest.raises(native.VrcError):
        native.grid_order(cam, (0, 1, 1), [])


def test_box_rect_is_conservative_and_tight(lib, orc):
    # No pixel outside the rectangle has a ray that meets the box; the rectangle exceeds the
    # bounding rectangle of the pixels whose rays do meet it by at most two pixels per side
    # (the one-pixel margin and the pixel a projected corner falls in; boxes wholly in front
    # of a perspective eye).
    rng = np.random.default_rng(5)
    dims = (64, 48, 40)
    checked = 0
    for cam in _cams(dims, 40, 30):
        for _ in range(6):
            a = rng.uniform(-0.5, np.array(dims) - 0.5)
            b = rng.uniform(-0.5, np.array(dims) - 0.5)
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            x0, y0, w, h = native.box_rect(cam, lo, hi)
            assert 0 <= x0 and 0 <= y0 and x0 + w <= cam.width and y0 + h <= cam.height
            hits = np.zeros((cam.height, cam.width), bool)
            for py in range(cam.height):
                for px in range(cam.width):
                    o, d, _, _, _ = orc.ray(cam, dims, px, py)
                    hits[py, px] = _interval(o, d, 0.0, np.inf, lo, hi) is not None
            inside = np.zeros_like(hits)
            inside[y0:y0 + h, x0:x0 + w] = True
            assert not (hits & ~inside).any()
            eye = np.array(cam.eye, np.float64)
            in_front = cam.ortho or all(
                np.dot(np.array(c) - eye, np.array(cam.center) - eye) > 0
                for c in [(u, v, s) for u in (lo[0], hi[0]) for v in (lo[1], hi[1])
                          for s in (lo[2], hi[2])])
            if hits.any() and in_front and not cam.ortho:
                ys, xs = np.nonzero(hits)
                assert x0 >= xs.min() - 2 and x0 + w - 1 <= xs.max() + 2
                assert y0 >= ys.min() - 2 and y0 + h - 1 <= ys.max() + 2
                checked += 1
    assert checked > 10


def test_box_rect_edge_cases(lib):
    dims = (32, 32, 32)
    cam = synth.orbit_cameras(2, 1, dims, 16, 12)[0]
    assert native.box_rect(cam, (5, 5, 5), (5, 9, 9)) == (0, 0, 0, 0)  # empty box
    inside = synth.Camera(0, (16.0, 16.0, 16.0), (40.0, 16.0, 16.0), (0.0, 1.0, 0.0), 60.0,
                          (0.0, 0.0), 16, 12)
    assert native.box_rect(inside, (0, 0, 0), (32, 32, 32)) == (0, 0, 16, 12)  # eye inside
    behind = synth.Camera(0, (16.0, 16.0, -50.0), (16.0, 16.0, -100.0), (0.0, 1.0, 0.0),
                          30.0, (0.0, 0.0), 16, 12)
    x0, y0, w, h = native.box_rect(behind, (0, 0, 0), (32, 32, 32))
    assert (x0, y0, w, h) == (0, 0, 16, 12)  # behind the eye: the whole image, conservatively
    with pytest.raises(native.VrcError):
        native.box_rect(synth.Camera(0, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), (0.0, 1.0, 0.0),
                                     30.0, (0.0, 0.0), 16, 12), (0, 0, 0), (1, 1, 1))
