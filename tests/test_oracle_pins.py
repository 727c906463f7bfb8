"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test states what fixes the expected value: the cubic B-spline's textbook definition and
moments, closed forms of the emission-absorption integral (Beer-Lambert, constant media),
geometric chord lengths, brute force on tiny inputs (an independent NumPy caster written as a
kernel sum), and the invariants the method guarantees (empty-space leaping changes no pixel,
early termination is bounded by the transmittance left).
"""
import math

import numpy as np
import pytest

from oracle import mini
from paper_2005_01442_gb300 import synth


# ----------------------------------------------------------------- resampling (a5)

def test_bspline_weights_match_textbook_kernel(orc):
    # The four weights at fraction f are the centred cubic B-spline at distances 1+f, f,
    # 1-f, 2-f (kernel written piecewise in oracle/mini.py, independent of the polynomials).
    for f in np.linspace(0.0, 1.0, 101, endpoint=False):
        w = orc.bspline_weights(f)
        ref = mini.beta3(np.array([1.0 + f, f, 1.0 - f, 2.0 - f]))
        np.testing.assert_allclose(w, ref, atol=1e-15)
        assert abs(w.sum() - 1.0) < 1e-15  # partition of unity
        assert np.all(w >= 0.0)


def test_bspline_weight_derivatives(orc):
    h = 1e-6
    for f in np.linspace(0.05, 0.95, 19):
        fd = (orc.bspline_weights(f + h) - orc.bspline_weights(f - h)) / (2 * h)
        np.testing.assert_allclose(orc.bspline_dweights(f), fd, atol=1e-8)
        assert abs(orc.bspline_dweights(f).sum()) < 1e-14


@pytest.mark.parametrize("dtype,val", [(np.uint16, 1234), (np.int16, -777), (np.float32, 3.25)])
def test_constant_field_is_reproduced(orc, dtype, val):
    vol = np.full((7, 9, 11), val, dtype)
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = rng.uniform(-0.5, [10.5, 8.5, 6.5])  # anywhere in the box, edges included
        assert abs(orc.sample(vol, p) - float(val)) <= 1e-12 * max(1.0, abs(float(val)))


def test_linear_field_is_reproduced_in_interior(orc):
    nz, ny, nx = 9, 11, 13
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c, d = 3.0, -2.0, 5.0, 7.0
    vol = (a * x + b * y + c * z + d).astype(np.float32)
    rng = np.random.default_rng(1)
    for _ in range(100):
        p = rng.uniform([1.0, 1.0, 1.0], [nx - 2.0, ny - 2.0, nz - 2.0])
        ref = a * p[0] + b * p[1] + c * p[2] + d
        assert abs(orc.sample(vol, p) - ref) < 1e-9
    # clamping breaks it at the border, as expected for clamp-to-edge taps
    assert abs(orc.sample(vol, (0.0, 5.0, 4.0)) - (b * 5 + c * 4 + d)) > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quadratic_gains_bspline_variance(orc, axis):
    # sum_i beta3(x - i) i^2 = x^2 + 1/3 (the cubic B-spline has variance 4/12): on a
    # non-cubic grid this also catches a transposed axis.
    nz, ny, nx = 10, 12, 14
    grids = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coord = [grids[2], grids[1], grids[0]][axis]
    vol = (coord.astype(np.float64) ** 2).astype(np.float32)
    rng = np.random.default_rng(2 + axis)
    hi = [nx - 2.0, ny - 2.0, nz - 2.0]
    for _ in range(60):
        p = rng.uniform([1.0, 1.0, 1.0], hi)
        assert abs(orc.sample(vol, p) - (p[axis] ** 2 + 1.0 / 3.0)) < 1e-9


def test_bilinear_cross_term_is_reproduced(orc):
    nz, ny, nx = 8, 9, 10
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = (x * y - 2.0 * y * z).astype(np.float32)
    rng = np.random.default_rng(5)
    for _ in range(60):
        p = rng.uniform([1.0, 1.0, 1.0], [nx - 2.0, ny - 2.0, nz - 2.0])
        assert abs(orc.sample(vol, p) - (p[0] * p[1] - 2.0 * p[1] * p[2])) < 1e-9


# ------------------------------------- interpolation / classification variants (next 1)

def test_trilinear_reproduces_multilinear_fields_and_interpolates(orc):
    # Trilinear interpolation reproduces every function a + bx + cy + dz + exy + fyz + gxz +
    # hxyz exactly in the interior and passes through the voxel values.
    nz, ny, nx = 7, 9, 11
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda x, y, z: 3.0 + 0.5 * x - 2.0 * y + 1.5 * z + 0.25 * x * y - 0.75 * y * z \
        + 0.1 * x * z + 0.05 * x * y * z  # noqa: E731
    vol = f(x, y, z).astype(np.float64).astype(np.float32)
    rng = np.random.default_rng(8)
    for _ in range(80):
        p = rng.uniform([0.0, 0.0, 0.0], [nx - 1.0, ny - 1.0, nz - 1.0])
        assert abs(orc.sample_linear(vol, p) - f(*p)) < 1e-4 * max(1.0, abs(f(*p)))
    for _ in range(20):
        i, j, k = rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)
        assert orc.sample_linear(vol, (i, j, k)) == float(vol[k, j, i])


def test_trilinear_matches_tent_kernel_sum_with_clamping(orc):
    # the tent-kernel sum over the edge-extended grid (NumPy), including points outside
    # the voxel grid where taps are clamped
    rng = np.random.default_rng(9)
    vol = rng.normal(0, 1, (5, 6, 7)).astype(np.float32)
    field = mini.Field(vol, "linear")
    for _ in range(100):
        p = rng.uniform([-0.5, -0.5, -0.5], [6.5, 5.5, 4.5])
        assert abs(orc.sample_linear(vol, p) - field(p)) < 1e-12


def test_preclassification_equals_post_for_an_affine_table(orc):
    # With a table affine in the index and values inside the window, classification commutes
    # with any interpolation whose weights sum to one: pre == post, cubic and trilinear.
    k = np.arange(256, dtype=np.float64)
    tf = np.stack([0.1 + 0.003 * k, 0.9 - 0.002 * k, 0.2 + 0.001 * k, 0.001 + 0.0015 * k],
                  -1).astype(np.float32)
    rng = np.random.default_rng(10)
    vol = rng.uniform(100, 3900, (6, 7, 8)).astype(np.float32)
    for interp in (0, 1):
        for _ in range(40):
            p = rng.uniform([1.0, 1.0, 1.0], [6.0, 5.0, 4.0])
            post = orc.sample_rgba(vol, p, tf, 0.0, 4095.0, interp, 0)
            pre = orc.sample_rgba(vol, p, tf, 0.0, 4095.0, interp, 1)
            np.testing.assert_allclose(pre, post, atol=1e-7)
    # ... and differs for a table with a step (the variants are not the same method)
    tf2 = tf.copy()
    tf2[128:, 3] = 0.9
    p = (3.3, 3.1, 2.7)
    assert np.abs(orc.sample_rgba(vol, p, tf2, 0.0, 4095.0, 0, 1)
                  - orc.sample_rgba(vol, p, tf2, 0.0, 4095.0, 0, 0)).max() > 1e-3


@pytest.mark.parametrize("interp,preclass", [(1, 0), (0, 1), (1, 1)])
def test_variant_renders_match_kernel_sum_brute_force(orc, interp, preclass):
    rng = np.random.default_rng(12)
    vol = rng.integers(0, 4096, (7, 8, 6)).astype(np.uint16)
    tf = synth.tf_random(5, 6)
    tf[:, 3] *= 0.6
    nz, ny, nx = vol.shape
    for cam in _cams_tiny((nx, ny, nz)):
        for step, ert in [(0.5, 1.0), (0.41, 0.6)]:
            a = orc.render(vol, tf, 0.0, 4095.0, cam, step, ert=ert, interp=interp,
                           preclass=preclass)
            b = mini.render(vol, tf, 0.0, 4095.0, cam, step, ert=ert, interp=interp,
                            preclass=preclass)
            assert np.abs(a - b).max() < 1e-11


@pytest.mark.parametrize("interp,preclass", [(1, 0), (0, 1), (1, 1)])
def test_variant_renders_unchanged_by_leaping(orc, interp, preclass):
    vol = synth.ct_volume((30, 34, 38), seed=13)
    tf = synth.tf_ct()
    cam = synth.orbit_cameras(17, 1, synth.dims_of(vol), 12, 10)[0]
    ref = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, interp=interp,
                     preclass=preclass)
    for B in (4, 8):
        img, (nom, ex) = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, brick=B,
                                    interp=interp, preclass=preclass, return_counts=True)
        assert np.array_equal(img, ref) and ex < nom


# ------------------------------------------------------ shading (the next row 2)

def test_bspline_gradient_is_exact_for_linear_and_quadratic_fields(orc):
    nz, ny, nx = 9, 10, 11
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = (2.0 + 1.5 * x - 0.75 * y + 0.5 * z).astype(np.float32)
    quad = (0.5 * x * x + y * z).astype(np.float32)
    rng = np.random.default_rng(21)
    for _ in range(40):
        p = rng.uniform([2.0, 2.0, 2.0], [nx - 3.0, ny - 3.0, nz - 3.0])
        np.testing.assert_allclose(orc.gradient(lin, p), [1.5, -0.75, 0.5], atol=1e-10)
        # x^2/2 -> (x^2 + 1/3)/2 and yz -> yz under the cubic B-spline: gradient (x, z, y)
        np.testing.assert_allclose(orc.gradient(quad, p), [p[0], p[2], p[1]], atol=1e-9)


def test_bspline_gradient_matches_differences_and_kernel_sum(orc):
    rng = np.random.default_rng(22)
    vol = rng.normal(0, 100, (7, 8, 9)).astype(np.float32)
    field = mini.Field(vol)
    h = 1e-5
    for _ in range(30):
        p = rng.uniform([-0.4, -0.4, -0.4], [8.4, 7.4, 6.4])
        g = orc.gradient(vol, p)
        np.testing.assert_allclose(g, field.gradient(p), atol=1e-9)
        fd = [(orc.sample(vol, p + h * e) - orc.sample(vol, p - h * e)) / (2 * h)
              for e in np.eye(3)]
        np.testing.assert_allclose(g, fd, atol=1e-4)


def test_phong_closed_forms(orc):
    # ortho view along +z (light and view along -z); constant table colour and opacity
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = (0.8, 0.5, 0.2)
    tf[:, 3] = 0.05
    ka, kd, ks, shin = 0.3, 0.7, 0.4, 8.0
    n = 20
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cam = synth.ortho_z_camera((n, n, n), 6, 6)
    lo, hi = -100.0, 4000.0
    # ramp along x: gradient normal to the view, n.L = 0: colour scaled by ka, opacity kept
    vol = (100.0 + 40.0 * x).astype(np.float32)
    plain = orc.render(vol, tf, lo, hi, cam, 0.5)
    lit = orc.render(vol, tf, lo, hi, cam, 0.5, phong=(ka, kd, ks, shin))
    np.testing.assert_allclose(lit[..., :3], ka * plain[..., :3], atol=1e-12)
    np.testing.assert_allclose(lit[..., 3], plain[..., 3], atol=1e-15)
    # ramp along z (slope 40 per voxel), opaque only for values 300..700, i.e. away from the
    # clamped first and last layers: every contributing sample has n.L = 40 / sqrt(40^2 +
    # eps^2), so the colour is the shaded table colour times the opacity
    vol = (100.0 + 40.0 * z).astype(np.float32)
    tf2 = tf.copy()
    tf2[:, 3] = 0.0
    tf2[26:49, 3] = 0.05
    eps = 0.01 * (hi - lo)
    nl = 40.0 / math.sqrt(40.0 ** 2 + eps ** 2)
    lit = orc.render(vol, tf2, lo, hi, cam, 0.5, phong=(ka, kd, ks, shin))
    ref = orc.render(vol, tf2, lo, hi, cam, 0.5)
    rgb = np.array([0.8, 0.5, 0.2])
    assert ref[..., 3].min() > 0.1
    np.testing.assert_array_equal(lit[..., 3], ref[..., 3])
    want = (rgb * (ka + kd * nl) + ks * nl ** shin)[None, None, :] * ref[..., 3:4]
    np.testing.assert_allclose(lit[..., :3], want, atol=1e-12)


def test_phong_render_matches_kernel_sum_brute_force(orc):
    rng = np.random.default_rng(23)
    vol = rng.integers(0, 4096, (7, 8, 6)).astype(np.uint16)
    tf = synth.tf_random(5, 6)
    tf[:, 3] *= 0.6
    nz, ny, nx = vol.shape
    ph = (0.25, 0.6, 0.3, 12.0)
    for cam in _cams_tiny((nx, ny, nz)):
        a = orc.render(vol, tf, 0.0, 4095.0, cam, 0.45, ert=0.7, phong=ph)
        b = mini.render(vol, tf, 0.0, 4095.0, cam, 0.45, ert=0.7, phong=ph)
        assert np.abs(a - b).max() < 1e-11


def test_phong_unchanged_by_leaping(orc):
    vol = synth.ct_volume((30, 34, 38), seed=24)
    tf = synth.tf_ct()
    cam = synth.orbit_cameras(25, 1, synth.dims_of(vol), 12, 10)[0]
    ph = (0.3, 0.7, 0.2, 16.0)
    ref = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, phong=ph)
    for B in (4, 8):
        assert np.array_equal(orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, brick=B,
                                         phong=ph), ref)


# ------------------------------------------- pre-integrated classification (next row 3)

def test_preint_table_closed_forms_and_brute_force(orc):
    # constant table: every entry is the constant medium over ds; a random table against the
    # vectorised NumPy rule and an entry-by-entry Python loop
    tf = np.zeros((256, 4), np.float32)
    tf[:] = (0.6, 0.3, 0.9, 0.2)
    tab = orc.preint_table(tf, 0.5)
    a = 1.0 - (1.0 - np.float64(np.float32(0.2))) ** 0.5
    np.testing.assert_allclose(tab[..., 3], a, atol=1e-15)
    np.testing.assert_allclose(tab[..., :3],
                               np.broadcast_to(np.array([0.6, 0.3, 0.9], np.float32) * a,
                                               tab[..., :3].shape), atol=1e-15)
    tf = synth.tf_random(31, 6)
    tab = orc.preint_table(tf, 0.37)
    np.testing.assert_allclose(tab, mini.preint_table(tf, 0.37), atol=1e-13)
    for i, k in [(0, 255), (17, 201), (200, 3), (128, 128)]:
        col, trans = np.zeros(3), 1.0
        for n in range(32):
            u = i + (k - i) * (n + 0.5) / 32
            i0 = min(int(math.floor(u)), 254)
            f = u - i0
            rgba = (1 - f) * tf[i0].astype(np.float64) + f * tf[i0 + 1].astype(np.float64)
            al = 1.0 - (1.0 - min(max(rgba[3], 0.0), 1.0 - 2.0 ** -24)) ** (0.37 / 32)
            col += trans * al * rgba[:3]
            trans *= 1.0 - al
        np.testing.assert_allclose(tab[i, k], np.append(col, 1.0 - trans), atol=1e-14)


def test_preint_constant_medium_spans_first_to_last_sample(orc):
    # a constant volume and table: each slab is the constant medium over the distance between
    # its two samples, so the opacity is that of the length from the first to the last sample
    n = 16
    vol = np.full((n, n, n), 1000, np.uint16)
    tf = np.zeros((256, 4), np.float32)
    tf[:] = (0.2, 0.7, 0.4, 0.1)
    cam = synth.ortho_z_camera((n, n, n), 4, 4)  # rays along z through 16 voxels
    img = orc.render(vol, tf, 0.0, 4095.0, cam, 0.5, preint=1)
    length = 16.0 - 0.5  # 32 segments of 0.5: midpoints 0.25 .. 15.75 from the entry
    a = np.float64(np.float32(0.1))
    np.testing.assert_allclose(img[..., 3], 1.0 - (1.0 - a) ** length, atol=1e-12)
    np.testing.assert_allclose(img[..., :3], np.array([0.2, 0.7, 0.4], np.float32) * img[..., 3:4],
                               atol=1e-12)


def test_preint_catches_a_thin_feature_that_sampling_misses(orc):
    # a ramp of 100 values per voxel sampled every half voxel (u jumps ~3.1 entries per
    # sample) and a table opaque only around one entry: samples step over it, slabs do not
    n = 24
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vol = (200 + 100 * z).astype(np.uint16)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 1.0
    tf[100, 3] = 0.9
    cam = synth.ortho_z_camera((n, n, n), 3, 3)
    post = orc.render(vol, tf, 0.0, 4095.0, cam, 0.5)
    pre = orc.render(vol, tf, 0.0, 4095.0, cam, 0.5, preint=1)
    assert pre[..., 3].min() > 5.0 * post[..., 3].max() and pre[..., 3].min() > 0.01


def test_preint_render_matches_numpy_brute_force(orc):
    rng = np.random.default_rng(32)
    vol = rng.integers(0, 4096, (7, 8, 6)).astype(np.uint16)
    tf = synth.tf_random(5, 6)
    tf[:, 3] *= 0.6
    nz, ny, nx = vol.shape
    for cam in _cams_tiny((nx, ny, nz)):
        for step, ert in [(0.5, 1.0), (0.43, 0.6)]:
            a = orc.render(vol, tf, 0.0, 4095.0, cam, step, ert=ert, preint=1)
            b = mini.render(vol, tf, 0.0, 4095.0, cam, step, ert=ert, preint=1)
            assert np.abs(a - b).max() < 1e-11


# ------------------------------------------------ whole path vs brute force (a3-a9)

def _cams_tiny(dims):
    nx, ny, nz = dims
    cams = [synth.ortho_z_camera(dims, 4, 4)]
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2)
    for eye in [(c[0] + 3.1, c[1] - 2.3, -14.0), (-11.0, c[1] + 1.7, c[2] + 9.0)]:
        cams.append(synth.Camera(0, eye, c, (0.0, 1.0, 0.0), 40.0, (0.0, 0.0), 4, 4).as_float32())
    return cams


@pytest.mark.parametrize("kind", ["u16", "f32"])
def test_oracle_matches_kernel_sum_brute_force(orc, kind):
    rng = np.random.default_rng(11)
    if kind == "u16":
        vol = rng.integers(0, 4096, (8, 8, 8)).astype(np.uint16)
        lo, hi = 0.0, 4095.0
    else:
        vol = rng.normal(0.0, 1.0, (8, 7, 6)).astype(np.float32)
        lo, hi = -2.0, 2.5
    tf = synth.tf_random(5, 6)
    tf[:, 3] *= 0.6
    nz, ny, nx = vol.shape
    for cam in _cams_tiny((nx, ny, nz)):
        for step, ert in [(0.5, 1.0), (0.37, 1.0), (0.5, 0.6)]:
            a = orc.render(vol, tf, lo, hi, cam, step, ert=ert)
            b = mini.render(vol, tf, lo, hi, cam, step, ert=ert)
            assert np.abs(a - b).max() < 1e-11


def test_ray_hits_box_where_expected(orc):
    cam = synth.ortho_z_camera((64, 64, 64), 128, 128)
    o, d, t0, t1, hit = orc.ray(cam, (64, 64, 64), 0, 0)
    assert hit and np.allclose(o, [-0.25, -0.25, -0.5]) and np.allclose(d, [0, 0, 1])
    assert t0 == 0.0 and t1 == 64.0
    o, d, _, _, _ = orc.ray(cam, (64, 64, 64), 127, 5)
    assert np.allclose(o[:2], [(127 + 0.5) * 0.5 - 0.5, (5 + 0.5) * 0.5 - 0.5])


def test_phantom_config_sample_count(orc):
    vol = synth.phantom()
    cam = synth.ortho_z_camera((64, 64, 64), 128, 128)
    _, counts = orc.render(vol, synth.tf_random(2), 0, 4095, cam, 0.5, return_counts=True)
    assert counts == (128 * 128 * 128, 128 * 128 * 128)  # 16384 rays x 128 samples


# ------------------------------------------------------------ closed forms (a6-a8)

def _flat_tf(rgba):
    return np.tile(np.asarray(rgba, np.float32), (256, 1))


@pytest.mark.parametrize("nz,step", [(64, 0.5), (10, 0.3), (17, 0.7), (33, 0.45)])
def test_constant_medium_closed_form(orc, nz, step):
    rgba = (0.8, 0.3, 0.55, 0.07)
    vol = np.full((nz, 6, 5), 100, np.uint16)
    cam = synth.ortho_z_camera((5, 6, nz), 3, 3)
    img = orc.render(vol, _flat_tf(rgba), 0, 4095, cam, step)
    a = np.float64(np.float32(rgba[3]))
    A = 1.0 - (1.0 - a) ** nz  # chord L = nz exactly
    assert np.allclose(img[..., 3], A, atol=1e-13)
    for c in range(3):
        assert np.allclose(img[..., c], np.float64(np.float32(rgba[c])) * A, atol=1e-13)


@pytest.mark.parametrize("step", [0.5, 0.3, 0.77])
def test_beer_lambert_oblique_and_perspective(orc, step):
    a = 0.02
    sigma = -math.log1p(-np.float64(np.float32(a)))
    n = 24
    vol = np.full((n, n, n), 7, np.uint16)
    tf = _flat_tf((1.0, 1.0, 1.0, a))
    c = (n - 1) / 2
    # orthographic 1x1 along the x-y diagonal through the centre: chord n*sqrt(2)
    d = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    eye = np.array([c, c, c]) - 40.0 * d
    cam = synth.Camera(1, tuple(eye), (c, c, c), (0.0, 0.0, 1.0), 0.0, (1.0, 1.0), 1, 1).as_float32()
    o, dd, t0, t1, _ = orc.ray(cam, (n, n, n), 0, 0)
    img = orc.render(vol, tf, 0, 4095, cam, step)
    T = 1.0 - img[0, 0, 3]
    assert abs(T - math.exp(-sigma * (t1 - t0))) < 1e-12
    assert abs((t1 - t0) - n * math.sqrt(2)) < 1e-4  # eye rounded to float32
    # perspective 1x1 on the z axis: the single ray is the optical axis, chord n
    cam = synth.Camera(0, (c, c, -30.0), (c, c, c), (0.0, 1.0, 0.0), 20.0, (0, 0), 1, 1).as_float32()
    T = 1.0 - orc.render(vol, tf, 0, 4095, cam, step)[0, 0, 3]
    assert abs(T - math.exp(-sigma * n)) < 1e-12


def test_sphere_chord_analytic_indicator(orc):
    # Indicator of a ball (no resampling): -ln T / sigma is the chord 2 sqrt(r^2 - d^2) up to
    # one misassigned segment per boundary crossing.
    n, r = 64, 20.0
    step = 0.5
    a = 0.05
    sigma = -math.log1p(-np.float64(np.float32(a)))
    tf = np.zeros((256, 4), np.float32)
    tf[255] = (1.0, 1.0, 1.0, a)
    c = np.array([31.5, 31.5, 31.5])
    vol = np.zeros((n, n, n), np.float32)
    cam = synth.ortho_z_camera((n, n, n), 64, 64)
    img = orc.render(vol, tf, 0.0, 1.0, cam, step, ball=(c, r))
    xs = (np.arange(64) + 0.5) - 0.5  # pixel centre x (and y) for extent 64 over 64 px
    X, Y = np.meshgrid(xs, xs)
    dist = np.hypot(X - c[0], Y - c[1])
    T = 1.0 - img[..., 3]
    inside = dist < r - 1.0
    chord = 2.0 * np.sqrt(np.maximum(r * r - dist ** 2, 0.0))
    est = -np.log(T[inside]) / sigma
    assert np.all(np.abs(est - chord[inside]) <= 2 * step + 1e-9)
    assert np.all(T[dist > r + 1e-9] == 1.0)


@pytest.mark.slow
def test_voxelised_sphere_line_integral(orc):
    # Voxelised ball r = 40 through resampling, rays along z. With a tiny opacity per unit
    # value the optical depth is the line integral of the B-spline field; since beta3
    # integrates to one, that integral is the 2D B-spline blend of the voxel column sums
    # (brute force below), and it stays within a voxel of the true chord 2 sqrt(r^2 - d^2).
    n, r = 96, 40.0
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vol = (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) <= r * r).astype(np.float32)
    eps = 1e-6
    tf = synth.tf_from_control_points([0, 255], [[1, 1, 1, 0], [1, 1, 1, eps]])
    cam = synth.ortho_z_camera((n, n, n), 24, 24)
    img = orc.render(vol, tf, 0.0, 1.0, cam, 0.25)
    px = (np.arange(24) + 0.5) * n / 24 - 0.5
    X, Y = np.meshgrid(px, px)
    T = 1.0 - img[..., 3]
    depth = -np.log(T) / np.float64(np.float32(eps))
    colsum = vol.astype(np.float64).sum(axis=0)  # (ny, nx)
    grid = np.arange(n, dtype=np.float64)
    blend = np.array([[mini.beta3(yy - grid) @ colsum @ mini.beta3(xx - grid) for xx in px]
                      for yy in px])
    assert np.abs(depth - blend).max() < 1e-3
    dist = np.hypot(X - c, Y - c)
    sel = dist <= r - 2.0
    chord = 2.0 * np.sqrt(r * r - dist[sel] ** 2)
    assert np.abs(depth[sel] - chord).max() < 1.0
    assert abs((depth[sel] - chord).mean()) < 0.2


# ------------------------------------------------------------------ bricks (a1, a2)

def _bricks_brute(vol, B):
    nz, ny, nx = vol.shape
    nb = [(n + B - 1) // B for n in (nz, ny, nx)]
    mn = np.empty(nb, vol.dtype)
    mx = np.empty(nb, vol.dtype)
    for bz in range(nb[0]):
        for by in range(nb[1]):
            for bx in range(nb[2]):
                sl = vol[max(bz * B - 1, 0):bz * B + B + 2, max(by * B - 1, 0):by * B + B + 2,
                         max(bx * B - 1, 0):bx * B + B + 2]
                mn[bz, by, bx] = sl.min()
                mx[bz, by, bx] = sl.max()
    return mn, mx


@pytest.mark.parametrize("dtype", [np.uint16, np.int16, np.float32])
@pytest.mark.parametrize("B", [4, 8, 16])
def test_brick_table_matches_brute_force(orc, dtype, B):
    rng = np.random.default_rng(B)
    shape = (19, 23, 37)
    if dtype == np.float32:
        vol = rng.normal(0, 100, shape).astype(np.float32)
    else:
        info = np.iinfo(dtype)
        vol = rng.integers(info.min, info.max, shape, endpoint=True).astype(dtype)
    mn, mx = orc.bricks(vol, B)
    rmn, rmx = _bricks_brute(vol, B)
    assert np.array_equal(mn, rmn) and np.array_equal(mx, rmx)


def test_empty_bricks_have_zero_alpha_on_their_range(orc):
    vol = synth.ct_volume((40, 48, 56), seed=9)
    tf = synth.tf_ct()
    lo, hi = synth.CT_LO, synth.CT_HI
    for B in (4, 8, 16):
        mn, mx = orc.bricks(vol, B)
        occ = orc.occupancy(mn, mx, tf, lo, hi)
        assert 0 < occ.sum() < occ.size
        for i in np.flatnonzero(occ == 0):
            vals = np.linspace(float(mn.flat[i]), float(mx.flat[i]), 33)
            for v in vals:
                assert mini.tf_lookup(v, tf, lo, hi)[3] == 0.0
        # brute force of the same float32 decision
        du = np.float32(255.0) / (np.float32(hi) - np.float32(lo))
        ulo = np.clip((mn.astype(np.float32) - np.float32(lo)) * du, 0, 255)
        uhi = np.clip((mx.astype(np.float32) - np.float32(lo)) * du, 0, 255)
        k0 = np.maximum(np.floor(ulo).astype(int) - 1, 0)
        k1 = np.minimum(np.ceil(uhi).astype(int) + 1, 255)
        ref = np.array([(tf[a:b + 1, 3] > 0).any() for a, b in zip(k0.ravel(), k1.ravel())])
        assert np.array_equal(occ.ravel().astype(bool), ref)


def test_empty_brick_decision_is_conservative_per_value(orc):
    # Single-valued bricks (min = max = v) swept over every 12-bit value, a table with
    # isolated opaque entries: an empty verdict must leave TF alpha zero on the whole index
    # interval [u(v) - 1/2, u(v) + 1/2], the room the float32 resampling rounding may use.
    vals = np.arange(0, 4096, dtype=np.uint16)
    tf = np.zeros((256, 4), np.float32)
    for k in (3, 40, 41, 97, 200, 255):
        tf[k] = (1.0, 1.0, 1.0, 0.5)
    occ = orc.occupancy(vals, vals, tf, 0.0, 4095.0)
    assert 0 < occ.sum() < occ.size
    for v in vals[occ == 0]:
        u = float(v) / 4095.0 * 255.0
        for du in np.linspace(-0.5, 0.5, 11):
            s = (u + du) * 4095.0 / 255.0
            assert mini.tf_lookup(s, tf, 0.0, 4095.0)[3] == 0.0, (v, du)


def test_cell_mask_brute_force_and_sampled_alpha(orc):
    # Cell mask: brute force of the support min/max (taps c-1 .. c+2 clamped, written here
    # with NumPy edge padding) and the float32 index rule; then sample points in every
    # transparent cell (and its faces) resampled by the independent NumPy caster have alpha 0.
    rng = np.random.default_rng(12)
    vol = np.full((9, 11, 13), -1000, np.int16)                  # air
    vol[2:8, 1:9, 3:12] = rng.normal(40, 10, (6, 8, 9))           # soft tissue
    vol[5, 4, 6] = 1200                                           # bone voxel
    vol[3, 7, 10] = 180                                           # faint, near the 150 HU edge
    tf = synth.tf_ct()
    lo, hi = synth.CT_LO, synth.CT_HI
    m = orc.cellmask(vol, tf, lo, hi)
    nz, ny, nx = vol.shape
    assert m.shape == (nz + 1, ny + 1, nx + 1)
    padded = np.pad(vol.astype(np.float64), 2, mode="edge")  # voxel v at padded index v + 2
    du = np.float32(255.0) / (np.float32(hi) - np.float32(lo))
    ref = np.zeros_like(m)
    for cz in range(-1, nz):
        for cy in range(-1, ny):
            for cx in range(-1, nx):
                box = padded[cz + 1:cz + 5, cy + 1:cy + 5, cx + 1:cx + 5]
                u0 = np.clip((np.float32(box.min()) - np.float32(lo)) * du, 0, 255)
                u1 = np.clip((np.float32(box.max()) - np.float32(lo)) * du, 0, 255)
                k0, k1 = max(int(np.floor(u0)) - 1, 0), min(int(np.ceil(u1)) + 1, 255)
                ref[cz + 1, cy + 1, cx + 1] = (tf[k0:k1 + 1, 3] > 0).any()
    assert np.array_equal(m, ref)
    assert 0 < m.sum() < m.size
    field = mini.Field(vol)
    zeros = np.argwhere(m == 0)
    for cz, cy, cx in zeros[rng.choice(len(zeros), min(len(zeros), 150), replace=False)]:
        for f in rng.uniform(0, 1, (4, 3)).tolist() + [[0.0, 0.0, 0.0], [0.999, 0.999, 0.999]]:
            p = (cx - 1 + f[0], cy - 1 + f[1], cz - 1 + f[2])
            assert mini.tf_lookup(field(p), tf, lo, hi)[3] == 0.0, (cx, cy, cz, f)


def test_cell_mask_refines_brick_occupancy(orc):
    # A cell's taps lie in the apron of the brick holding the cell, so an empty brick holds
    # only transparent cells; and an isolated opaque voxel marks exactly the 4^3 cells whose
    # support contains it.
    vol = synth.ct_volume((24, 20, 28), seed=13)
    tf = synth.tf_ct()
    lo, hi = synth.CT_LO, synth.CT_HI
    m = orc.cellmask(vol, tf, lo, hi)
    for B in (4, 8):
        occ = orc.occupancy(*orc.bricks(vol, B), tf, lo, hi)
        nz, ny, nx = vol.shape
        for cz in range(-1, nz):
            for cy in range(-1, ny):
                for cx in range(-1, nx):
                    b = (max(cz, 0) // B, max(cy, 0) // B, max(cx, 0) // B)
                    if occ[b] == 0:
                        assert m[cz + 1, cy + 1, cx + 1] == 0
    flat = np.full((10, 10, 10), -1000, np.int16)
    flat[4, 5, 6] = 1200
    mf = orc.cellmask(flat, tf, lo, hi)
    expect = np.zeros_like(mf)
    expect[4 - 2 + 1:4 + 1 + 1 + 1, 5 - 2 + 1:5 + 1 + 1 + 1, 6 - 2 + 1:6 + 1 + 1 + 1] = 1
    assert np.array_equal(mf, expect)


# --------------------------------------------------------- ESL and ERT invariants (a4, a8)

def _ct_small():
    vol = synth.ct_volume((48, 64, 64), seed=21)
    return vol, synth.tf_ct(), synth.CT_LO, synth.CT_HI


def test_empty_space_leaping_changes_no_pixel(orc):
    vol, tf, lo, hi = _ct_small()
    dims = synth.dims_of(vol)
    for cam in synth.orbit_cameras(4, 3, dims, 48, 40):
        ref, cref = orc.render(vol, tf, lo, hi, cam, 0.5, return_counts=True)
        for B in (4, 8, 16):
            img, cnt = orc.render(vol, tf, lo, hi, cam, 0.5, brick=B, return_counts=True)
            assert np.array_equal(img, ref)
            assert cnt[0] == cref[0] and cnt[1] < cref[1]


def test_early_termination_bounded_by_remaining_transmittance(orc):
    vol, tf, lo, hi = _ct_small()
    tf = tf.copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 3.0, 0.95)
    dims = synth.dims_of(vol)
    for cam in synth.orbit_cameras(6, 2, dims, 48, 40):
        full = orc.render(vol, tf, lo, hi, cam, 0.5)
        ert = orc.render(vol, tf, lo, hi, cam, 0.5, ert=0.999, brick=8)
        t_stop = 1.0 - ert[..., 3]
        stopped = ert[..., 3] > 0.999
        assert stopped.any()
        diff = np.abs(full - ert).max(axis=-1)
        assert np.all(diff[stopped] <= t_stop[stopped] + 1e-15)
        assert np.array_equal(full[~stopped], ert[~stopped])


# ------------------------------------------------------------------- gradient (a10)

def test_gradient_closed_form_constant_volume(orc):
    # u lands exactly on entry k, so dA/dTF[k].alpha = L (1-a)^(L-1) and dC/dTF[k].rgb = A.
    nz, a = 12, 0.1
    vol = np.full((nz, 4, 4), 100.0, np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[100] = (0.2, 0.4, 0.6, a)
    cam = synth.ortho_z_camera((4, 4, nz), 2, 2)
    g = np.zeros((4, 4))
    g[:, 3] = 1.0
    gtf, _ = orc.render_grad(vol, tf, 0.0, 255.0, cam, 0.5, g)
    a64 = np.float64(np.float32(a))
    assert abs(gtf[100, 3] - 4 * nz * (1 - a64) ** (nz - 1)) < 1e-10
    g[:] = 0
    g[:, 0] = 1.0
    gtf, _ = orc.render_grad(vol, tf, 0.0, 255.0, cam, 0.5, g)
    assert abs(gtf[100, 0] - 4 * (1 - (1 - a64) ** nz)) < 1e-10


def test_gradient_at_zero_opacity_from_above(orc):
    """open_alpha: at a table opacity of exactly 0 the opacity correction's derivative is taken
    from above: for a constant medium dA/da = L (1-0)^(L-1) = L per ray, where the default
    (clamped side) gives 0; and for a CT scene it matches a one-sided forward difference of the
    forward render (Richardson-extrapolated, h and h/2) on entries whose opacity is 0."""
    nz = 12
    vol = np.full((nz, 4, 4), 100.0, np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[100] = (0.2, 0.4, 0.6, 0.0)
    cam = synth.ortho_z_camera((4, 4, nz), 2, 2)
    g = np.zeros((4, 4))
    g[:, 3] = 1.0
    shut, _ = orc.render_grad(vol, tf, 0.0, 255.0, cam, 0.5, g)
    opened, _ = orc.render_grad(vol, tf, 0.0, 255.0, cam, 0.5, g, open_alpha=True)
    assert shut[100, 3] == 0.0
    assert abs(opened[100, 3] - 4 * nz) < 1e-10
    with pytest.raises(ValueError):  # leaping would drop the samples that carry it
        orc.render_grad(vol, tf, 0.0, 255.0, cam, 0.5, g, brick=8, open_alpha=True)
    # a CT scene: entries below 150 HU are fully transparent in this table
    vol, tf, cam, g = _fd_setup()
    tf = synth.tf_ct(seed=4)
    gtf, _ = orc.render_grad(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, g, open_alpha=True)
    zero = np.flatnonzero((tf[:, 3] == 0.0) & (np.abs(gtf[:, 3]) > 1e-3 * np.abs(gtf[:, 3]).max()))
    assert zero.size >= 5
    rng = np.random.default_rng(19)
    base = _loss(orc, vol, tf, cam, g)
    for k in rng.permutation(zero)[:5]:
        def fwd(h):
            t = tf.copy()
            t[k, 3] = np.float32(h)
            return (_loss(orc, vol, t, cam, g) - base) / float(np.float32(h))
        fd = 2.0 * fwd(5e-5) - fwd(1e-4)
        assert abs(fd - gtf[k, 3]) <= 2e-3 * abs(gtf[k, 3]), (k, fd, gtf[k, 3])


def _fd_setup():
    vol = synth.ct_volume((24, 24, 24), seed=31).astype(np.float32)
    vol = vol + np.random.default_rng(3).normal(0, 30, vol.shape).astype(np.float32)
    tf = synth.tf_ct(seed=4)
    tf[:, 3] = np.maximum(tf[:, 3], 0.01)
    dims = synth.dims_of(vol)
    cam = synth.orbit_cameras(12, 1, dims, 12, 10)[0]
    g = np.random.default_rng(8).normal(0, 1, (cam.height * cam.width, 4))
    return vol, tf, cam, g


def _loss(orc, vol, tf, cam, g):
    img = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5)
    return float((img.reshape(-1, 4) * g).sum())


@pytest.mark.slow
def test_gradient_matches_central_differences(orc):
    vol, tf, cam, g = _fd_setup()
    gtf, gvol = orc.render_grad(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, g)
    rng = np.random.default_rng(17)
    h = 1e-3
    # TF entries used by the image (rgba is linear in the table, so no kinks)
    used = np.flatnonzero(np.abs(gtf).sum(1) > 1e-6)
    checked = 0
    for k in rng.permutation(used)[:25]:
        c = int(rng.integers(0, 4))
        tp, tm = tf.astype(np.float64).copy(), tf.astype(np.float64).copy()
        tp[k, c] += h
        tm[k, c] -= h
        # the oracle takes float32 tables: perturb in float64, hand over exact float32 values
        tp32, tm32 = tp.astype(np.float32), tm.astype(np.float32)
        step = float(tp32[k, c]) - float(tm32[k, c])
        fd = (_loss(orc, vol, tp32, cam, g) - _loss(orc, vol, tm32, cam, g)) / step
        if abs(gtf[k, c]) > 1e-4:
            assert abs(fd - gtf[k, c]) <= 1e-3 * abs(gtf[k, c]) + 1e-7
            checked += 1
    assert checked >= 10
    # voxels with a visible effect, skipping samples that sit on a TF kink (the FD at h and
    # at h/4 disagree there)
    cand = np.flatnonzero(np.abs(gvol).ravel() > 0.05 * np.abs(gvol).max())
    checked = 0
    for vi in rng.permutation(cand)[:40]:
        def fd_at(hh):
            vp, vm = vol.copy(), vol.copy()
            vp.flat[vi] += hh
            vm.flat[vi] -= hh
            hh_eff = (float(vp.flat[vi]) - float(vm.flat[vi])) / 2
            return (_loss(orc, vp, tf, cam, g) - _loss(orc, vm, tf, cam, g)) / (2 * hh_eff)
        hv = 1e-3 * max(1.0, abs(float(vol.flat[vi])))
        f1, f2 = fd_at(hv), fd_at(hv / 4)
        if abs(f1 - f2) > 1e-4 * abs(f1):
            continue  # kink inside the stencil
        assert abs(f1 - gvol.flat[vi]) <= 1e-3 * abs(gvol.flat[vi])
        checked += 1
        if checked >= 25:
            break
    assert checked >= 10


# ----------------------------------- object-order pieces and sort-last compositing (next 4)

def _cell_range_of_brick(b, B, n):
    return (-1 if b == 0 else b * B), min(b * B + B, n)


@pytest.mark.parametrize("v", [(6, 5, 4), (0, 0, 0), (12, 10, 8), (7, 3, 8)])
@pytest.mark.parametrize("B", [4, 8])
def test_brick_aabbs_single_voxel_closed_form(orc, v, B):
    # An isolated opaque voxel v in air opens exactly the cells c with max(v-2, -1) <= c <=
    # min(v+1, n-1) per axis (the cells whose clamped taps c-1 .. c+2 reach v); a brick's box
    # is that range cut to the brick's own cells, and every other brick's box is empty.
    nx, ny, nz = 13, 11, 9
    vol = np.full((nz, ny, nx), -1000, np.int16)
    vol[v[2], v[1], v[0]] = 1200
    box = orc.brick_aabbs(vol, synth.tf_ct(), synth.CT_LO, synth.CT_HI, B)
    n = (nx, ny, nz)
    nb = [(k + B - 1) // B for k in n]
    assert box.shape == (nb[2], nb[1], nb[0], 6) and box.dtype == np.int16
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                b = (bx, by, bz)
                lo, hi = [], []
                for k in range(3):
                    c0, c1 = _cell_range_of_brick(b[k], B, n[k])
                    lo.append(max(c0, v[k] - 2, -1))
                    hi.append(min(c1, v[k] + 2, n[k]))
                if all(hi[k] > lo[k] for k in range(3)):
                    assert box[bz, by, bx].tolist() == lo + hi, b
                else:
                    assert not box[bz, by, bx].any(), b


def test_brick_aabbs_are_the_bounding_boxes_of_open_cells(orc):
    # Brute force with NumPy on a small CT-like volume: each occupied brick's box is the
    # bounding box of its open cells; boxes of bricks without open cells (and of empty
    # bricks) are zero.
    rng = np.random.default_rng(31)
    vol = np.full((20, 18, 22), -1000, np.int16)                 # air
    vol[3:11, 2:12, 4:17] = rng.normal(40, 10, (8, 10, 13))       # soft tissue
    vol[14, 13, 18] = 1200                                        # bone voxel
    tf, lo, hi = synth.tf_ct(), synth.CT_LO, synth.CT_HI
    m = orc.cellmask(vol, tf, lo, hi)
    nz, ny, nx = vol.shape
    for B in (4, 8):
        occ = orc.occupancy(*orc.bricks(vol, B), tf, lo, hi)
        box = orc.brick_aabbs(vol, tf, lo, hi, B)
        cells = np.argwhere(m == 1) - 1  # (cz, cy, cx) cell coordinates
        bidx = np.maximum(cells, 0) // B
        seen = tighter = 0
        for bz, by, bx in np.ndindex(occ.shape):
            sel = cells[(bidx[:, 0] == bz) & (bidx[:, 1] == by) & (bidx[:, 2] == bx)]
            if occ[bz, by, bx] == 0 or len(sel) == 0:
                assert not box[bz, by, bx].any()
                continue
            seen += 1
            mn, mx = sel.min(axis=0)[::-1], sel.max(axis=0)[::-1] + 1  # to (x, y, z)
            assert box[bz, by, bx].tolist() == mn.tolist() + mx.tolist()
            c0 = [_cell_range_of_brick(b, B, n)[0] for b, n in zip((bx, by, bz), (nx, ny, nz))]
            c1 = [_cell_range_of_brick(b, B, n)[1] for b, n in zip((bx, by, bz), (nx, ny, nz))]
            tighter += mn.tolist() != c0 or mx.tolist() != c1
        assert 0 < seen < occ.size and tighter > 0


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 2, 2), (3, 1, 2), (4, 3, 1)])
def test_piece_grid_tiles_bricks_and_cells_once(orc, grid):
    # The pieces of a grid cover every brick once, and their cell ranges cover the cells
    # -1 .. n-1 of each axis once (the decomposition neither drops nor repeats a sample).
    dims, B = (37, 29, 20), 4
    nb = [(n + B - 1) // B for n in dims]
    pieces = orc.piece_grid(dims, B, grid)
    assert len(pieces) == grid[0] * grid[1] * grid[2]
    count = np.zeros(nb[::-1], np.int32)
    ccount = np.zeros([n + 1 for n in dims[::-1]], np.int32)
    for blo, bhi in pieces:
        assert all(bhi[k] > blo[k] for k in range(3))
        count[blo[2]:bhi[2], blo[1]:bhi[1], blo[0]:bhi[0]] += 1
        clo, chi = orc.piece_cells(dims, B, blo, bhi)
        ccount[clo[2] + 1:chi[2] + 1, clo[1] + 1:chi[1] + 1, clo[0] + 1:chi[0] + 1] += 1
    assert (count == 1).all() and (ccount == 1).all()


def _tiny_piece_scene():
    vol = synth.ct_volume((12, 14, 16), seed=33)
    tf = synth.tf_ct().copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 4.0, 0.9)
    return vol, tf, synth.CT_LO, synth.CT_HI


@pytest.mark.parametrize("ert", [1.0, 0.9])
def test_piece_partial_matches_brute_force(orc, ert):
    # A piece's partial image is the brute-force caster with every sample outside the
    # piece's bricks dropped (NumPy rays, segments and kernel sum), its own early termination
    # included.
    vol, tf, lo, hi = _tiny_piece_scene()
    dims = synth.dims_of(vol)
    B = 4
    cam = synth.orbit_cameras(1, 9, dims, 10, 8)[0]
    for blo, bhi in orc.piece_grid(dims, B, (2, 2, 1))[1:3]:
        def keep(p, blo=blo, bhi=bhi):
            b = [max(int(math.floor(p[k])), 0) // B for k in range(3)]
            return all(blo[k] <= b[k] < bhi[k] for k in range(3))
        ref = mini.render(vol, tf, lo, hi, cam, 0.7, ert=ert, keep=keep)
        got = orc.render_piece(vol, tf, lo, hi, cam, 0.7, B, blo, bhi, ert=ert)
        assert np.abs(got - ref).max() < 1e-9
        assert ref[..., 3].max() > 0.05


@pytest.mark.parametrize("grid", [(2, 2, 2), (3, 1, 2)])
def test_sort_last_composite_equals_one_pass_render(orc, grid):
    # The over operator is associative: composited in the order each ray meets the pieces,
    # the partial images of all pieces give the one-pass render (no early termination) to
    # rounding, for perspective and orthographic views. Reversed, they do not.
    vol, tf, lo, hi = _ct_small()
    dims = synth.dims_of(vol)
    B = 8
    cams = list(synth.orbit_cameras(2, 5, dims, 24, 20)) + [synth.ortho_z_camera(dims, 24, 20)]
    pieces = orc.piece_grid(dims, B, grid)
    boxes = [orc.piece_cells(dims, B, blo, bhi) for blo, bhi in pieces]
    for cam in cams:
        pix = [(x, y) for y in range(cam.height) for x in range(cam.width)]
        full = orc.render(vol, tf, lo, hi, cam, 0.5, brick=B).reshape(-1, 4)
        parts = np.stack([orc.render_piece(vol, tf, lo, hi, cam, 0.5, B, blo, bhi).reshape(-1, 4)
                          for blo, bhi in pieces])
        order = orc.pixel_piece_order(cam, dims, boxes, pix)
        comp = orc.composite(parts, order)
        assert np.abs(comp - full).max() < 1e-12
        assert full[:, 3].max() > 0.5
        wrong = orc.composite(parts, order[:, ::-1])
        assert np.abs(wrong - full).max() > 1e-3
