"""GPU parity of object-order rendering (pieces of whole bricks, sort-last compositing) against
the FP64 oracle, through the C ABI.

Bars: tight brick boxes and plan geometry bit-exact; piece partial images and blended images
within max |d| <= 1e-4 per RGBA channel of the oracle (pixels whose early termination sits
within 1e-5 of the threshold in some piece held to 2e-3, as in the one-pass tests); the
rectangle a piece renders loses no pixel of its full-image partial; without early
termination the blended image equals the one-pass render to float32 rounding.
"""
import numpy as np
import pytest

from paper_2005_01442_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
ERT_MARGIN = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def R(torch):
    from paper_2005_01442_gb300 import build
    from paper_2005_01442_gb300.renderer import Renderer
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def _air_tissue(seed=31, shape=(37, 45, 50)):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    vol = np.full(shape, -1000, np.int16)
    vol[4:nz // 2, 3:ny - 10, 6:nx - 12] = rng.normal(60, 25, (nz // 2 - 4, ny - 13, nx - 18))
    vol[nz - 6, ny - 5, nx - 4] = 1500
    return vol


def _scene(R, vol, B, tf=None):
    vid = R.upload_volume(vol)
    R.build_bricks(vid, B)
    tf = synth.tf_ct() if tf is None else tf
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    return vid, tid, tf


def _dims(vol):
    return synth.dims_of(vol)


# ------------------------------------------------------------------ exact tables and plans

@pytest.mark.parametrize("B", [8, 16])
@pytest.mark.parametrize("which", ["ct", "air"])
def test_brick_boxes_bit_exact(R, orc, B, which):
    vol = synth.ct_volume((45, 50, 61), seed=22) if which == "ct" else _air_tissue()
    vid, tid, tf = _scene(R, vol, B)
    got = R.aabbs(vid, tid, B)
    ref = orc.brick_aabbs(vol, tf, synth.CT_LO, synth.CT_HI, B)
    assert got.shape == ref.shape and np.array_equal(got, ref)
    assert (ref[..., 3] > ref[..., 0]).any()
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 2, 2), (3, 2, 1), (4, 1, 3)])
def test_plan_geometry_matches_oracle(R, orc, grid):
    vol = _air_tissue()
    B = 8
    vid, tid, tf = _scene(R, vol, B)
    plan = R.build_pieces(vid, tid, B, grid)
    pieces, cuts = R.pieces(plan)
    dims = _dims(vol)
    ref = orc.piece_grid(dims, B, grid)
    boxes = orc.brick_aabbs(vol, tf, synth.CT_LO, synth.CT_HI, B)
    assert len(pieces) == len(ref)
    for p, (blo, bhi) in zip(pieces, ref):
        assert p["brick_lo"] == blo and p["brick_hi"] == bhi
        clo, chi = orc.piece_cells(dims, B, blo, bhi)
        assert p["cell_lo"] == clo and p["cell_hi"] == chi
        sub = boxes[blo[2]:bhi[2], blo[1]:bhi[1], blo[0]:bhi[0]].reshape(-1, 6).astype(int)
        sub = sub[sub[:, 3] > sub[:, 0]]
        if len(sub) == 0:
            assert p["vis_lo"] == (0, 0, 0) and p["vis_hi"] == (0, 0, 0)
        else:
            assert p["vis_lo"] == tuple(sub[:, :3].min(axis=0))
            assert p["vis_hi"] == tuple(sub[:, 3:].max(axis=0))
    expect_cuts = [float(c) for a in range(3) for c in sorted({pc[0][a] for pc in
                   [orc.piece_cells(dims, B, lo, hi) for lo, hi in ref]})[1:]]
    assert cuts == expect_cuts
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


# ----------------------------------------------------------------- piece partial images

@pytest.mark.parametrize("kernel", [0, 1, 4])
@pytest.mark.parametrize("ert", [1.0, 0.999])
def test_piece_partials_match_oracle(R, orc, torch, kernel, ert):
    vol = synth.ct_volume((48, 64, 72), seed=23)
    B = 8
    tf = synth.tf_ct().copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 3.0, 0.95)
    vid, tid, _ = _scene(R, vol, B, tf)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, (2, 2, 2))
    pieces, _ = R.pieces(plan)
    cam = synth.orbit_cameras(5, 1, dims, 56, 44)[0]
    for k in (0, 3, 6):
        p = pieces[k]
        img = R.render_piece(plan, k, cam, (0, 0, cam.width, cam.height), 0.5, ert, B,
                             kernel=kernel)
        ref, mg = orc.render_piece(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, B,
                                   p["brick_lo"], p["brick_hi"], ert=ert, return_margin=True)
        d = np.abs(img.cpu().numpy().astype(np.float64) - ref).max(axis=-1)
        flagged = mg < ERT_MARGIN
        assert d[~flagged].max(initial=0.0) <= TOL, (k, d.max())
        assert d[flagged].max(initial=0.0) <= 2e-3
        assert ref[..., 3].max() > 0.1
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


def test_piece_rect_loses_nothing_and_is_offset_exactly(R, orc, torch):
    # Rendered over the whole image, a piece's partial is (0, 0, 0, 0) outside the rectangle
    # of its visible box, and the rectangle render reproduces the inside bit for bit (same
    # rays through the pixel offset).
    from paper_2005_01442_gb300 import native
    vol = _air_tissue(shape=(48, 56, 64))
    B = 8
    vid, tid, _ = _scene(R, vol, B)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, (2, 2, 2))
    pieces, _ = R.pieces(plan)
    cams = list(synth.orbit_cameras(8, 3, dims, 80, 64)) + [synth.ortho_z_camera(dims, 80, 64)]
    shrunk = 0
    for cam in cams:
        for k, p in enumerate(pieces):
            lo = [max(float(p["vis_lo"][a]), -0.5) for a in range(3)]
            hi = [min(float(p["vis_hi"][a]), dims[a] - 0.5) for a in range(3)]
            x0, y0, w, h = native.box_rect(cam, lo, hi)
            full = R.render_piece(plan, k, cam, (0, 0, cam.width, cam.height), 0.5, 0.999, B)
            full = full.cpu().numpy()
            outside = np.ones(full.shape[:2], bool)
            outside[y0:y0 + h, x0:x0 + w] = False
            assert not full[outside].any(), (k, cam)
            shrunk += w * h < cam.width * cam.height
            if w and h:
                part = R.render_piece(plan, k, cam, (x0, y0, w, h), 0.5, 0.999, B).cpu().numpy()
                assert np.array_equal(part, full[y0:y0 + h, x0:x0 + w])
    assert shrunk > 0
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


# ------------------------------------------------------------------ sort-last compositing

@pytest.mark.parametrize("grid", [(2, 2, 2), (3, 1, 2)])
@pytest.mark.parametrize("ert", [1.0, 0.999])
def test_sortlast_matches_oracle_composite(R, orc, torch, grid, ert):
    # The blended image against the oracle's partials composited per pixel in the order its
    # ray enters the pieces (slab tests), an order the GPU path never computes.
    vol = synth.ct_volume((48, 64, 72), seed=24)
    B = 8
    tf = synth.tf_ct().copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 3.0, 0.95)
    vid, tid, _ = _scene(R, vol, B, tf)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, grid)
    pieces, _ = R.pieces(plan)
    boxes = [(p["cell_lo"], p["cell_hi"]) for p in pieces]
    cams = list(synth.orbit_cameras(9, 2, dims, 40, 32)) + [synth.ortho_z_camera(dims, 40, 32)]
    for cam in cams:
        img = R.render_sortlast(plan, cam, 0.5, ert, B).cpu().numpy().astype(np.float64)
        pix = [(x, y) for y in range(cam.height) for x in range(cam.width)]
        parts, flagged = [], np.zeros(len(pix), bool)
        for p in pieces:
            part, mg = orc.render_piece(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, B,
                                        p["brick_lo"], p["brick_hi"], ert=ert,
                                        return_margin=True)
            parts.append(part.reshape(-1, 4))
            flagged |= mg.reshape(-1) < ERT_MARGIN
        ref = orc.composite(np.stack(parts), orc.pixel_piece_order(cam, dims, boxes, pix))
        d = np.abs(img.reshape(-1, 4) - ref).max(axis=-1)
        assert d[~flagged].max(initial=0.0) <= TOL, d.max()
        assert d[flagged].max(initial=0.0) <= 2e-3
        assert ref[:, 3].max() > 0.5
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("variant", [{}, {"interp": 1}, {"preclass": 1},
                                     {"phong": (0.3, 0.6, 0.2, 16.0)}, {"kernel": 1}])
def test_sortlast_equals_one_pass_render_without_ert(R, torch, variant):
    vol = synth.ct_volume((64, 80, 96), seed=25)
    B = 8
    vid, tid, _ = _scene(R, vol, B)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, (3, 2, 2))
    for cam in list(synth.orbit_cameras(10, 3, dims, 96, 80)) + [synth.ortho_z_camera(dims, 96, 80)]:
        one = R.render(vid, tid, cam, 0.5, 1.0, B, **variant).cpu().numpy()
        sl = R.render_sortlast(plan, cam, 0.5, 1.0, B, **variant).cpu().numpy()
        assert np.abs(sl - one).max() <= 2e-5, np.abs(sl - one).max()
        assert one[..., 3].max() > 0.5
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


def test_single_piece_is_the_one_pass_render(R, torch):
    vol = synth.ct_volume((48, 64, 72), seed=26)
    B = 16
    vid, tid, _ = _scene(R, vol, B)
    plan = R.build_pieces(vid, tid, B, (1, 1, 1))
    for cam in synth.orbit_cameras(11, 3, _dims(vol), 64, 48):
        one = R.render(vid, tid, cam, 0.5, 0.999, B).cpu().numpy()
        sl = R.render_sortlast(plan, cam, 0.5, 0.999, B).cpu().numpy()
        assert np.array_equal(sl[..., :3], one[..., :3])
        assert np.abs(sl[..., 3] - one[..., 3]).max() <= 1e-7
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


def test_invisible_pieces_are_skipped(R, orc, torch):
    # A transfer function that shows only the bone voxel leaves all but one piece without a
    # visible box; the blend still matches the oracle.
    vol = _air_tissue(shape=(40, 48, 56))
    vol[32:35, 40:43, 49:52] = 1500  # a bone blob (its spline reaches the bone range)
    B = 8
    tf = synth.tf_ct().copy()
    u_bone = (1000.0 - synth.CT_LO) / (synth.CT_HI - synth.CT_LO) * 255.0
    tf[: int(u_bone), 3] = 0.0
    vid, tid, _ = _scene(R, vol, B, tf)
    plan = R.build_pieces(vid, tid, B, (2, 2, 2))
    pieces, _ = R.pieces(plan)
    visible = [p for p in pieces if p["vis_hi"] != (0, 0, 0)]
    assert len(visible) == 1
    dims = _dims(vol)
    cam = synth.orbit_cameras(12, 1, dims, 48, 40)[0]
    img = R.render_sortlast(plan, cam, 0.5, 1.0, B).cpu().numpy()
    ref = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5)
    assert np.abs(img - ref).max() <= TOL
    assert ref[..., 3].max() > 0.05
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


# ------------------------------------------------------- ordered pass (front to back, ERT)

@pytest.mark.parametrize("grid", [(2, 2, 2), (3, 1, 2), (4, 4, 2)])
@pytest.mark.parametrize("ert", [1.0, 0.999])
def test_ordered_pass_matches_oracle_one_pass_render(R, orc, torch, grid, ert):
    # Pieces drawn front to back through one running image, rays terminating across them:
    # the one-pass image of the oracle, early termination included.
    vol = synth.ct_volume((48, 64, 72), seed=28)
    B = 8
    tf = synth.tf_ct().copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 3.0, 0.95)
    vid, tid, _ = _scene(R, vol, B, tf)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, grid)
    cams = list(synth.orbit_cameras(14, 2, dims, 48, 40)) + [synth.ortho_z_camera(dims, 48, 40)]
    for cam in cams:
        img = R.render_ordered(plan, cam, 0.5, ert, B).cpu().numpy().astype(np.float64)
        ref, mg = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=ert, brick=B,
                             return_margin=True)
        d = np.abs(img - ref).max(axis=-1)
        flagged = mg < ERT_MARGIN
        assert d[~flagged].max(initial=0.0) <= TOL, d.max()
        assert d[flagged].max(initial=0.0) <= 1e-3
        assert ref[..., 3].max() > 0.9
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("variant", [{}, {"interp": 1}, {"preclass": 1},
                                     {"phong": (0.3, 0.6, 0.2, 16.0)}, {"kernel": 1}])
def test_ordered_pass_equals_one_pass_render(R, torch, variant):
    vol = synth.ct_volume((64, 80, 96), seed=29)
    B = 8
    vid, tid, _ = _scene(R, vol, B)
    dims = _dims(vol)
    plan = R.build_pieces(vid, tid, B, (3, 2, 2))
    one_plan = R.build_pieces(vid, tid, B, (1, 1, 1))
    for cam in list(synth.orbit_cameras(15, 3, dims, 96, 80)) + [synth.ortho_z_camera(dims, 96, 80)]:
        for ert in (1.0, 0.999):
            one = R.render(vid, tid, cam, 0.5, ert, B, **variant).cpu().numpy()
            od = R.render_ordered(plan, cam, 0.5, ert, B, **variant).cpu().numpy()
            d = np.abs(od - one).max(axis=-1)
            # a ray whose opacity crosses the threshold within float rounding may stop one
            # sample apart (at most the termination bound)
            assert (d > 2e-5).mean() <= 1e-3 and d.max() <= 1e-3, d.max()
            single = R.render_ordered(one_plan, cam, 0.5, ert, B, **variant).cpu().numpy()
            assert np.array_equal(single, one)  # one piece: the one-pass render bit for bit
    R.free_pieces(plan)
    R.free_pieces(one_plan)
    R.free_volume(vid)
    R.free_tf(tid)


# --------------------------------------------------------------------------- rejections

def test_piece_calls_reject_bad_arguments(R, torch):
    from paper_2005_01442_gb300.native import VrcError
    vol = synth.ct_volume((32, 40, 48), seed=27)
    B = 8
    vid, tid, tf = _scene(R, vol, B)
    nb = [(n + B - 1) // B for n in _dims(vol)]
    with pytest.raises(VrcError):
        R.build_pieces(vid, tid, B, (nb[0] + 1, 1, 1))  # more pieces than bricks
    with pytest.raises(VrcError):
        R.build_pieces(vid, tid, B, (4, 4, 5))  # more than 64 pieces
    with pytest.raises(VrcError):
        R.build_pieces(vid, tid, 16, (1, 1, 1))  # brick table not built
    plan = R.build_pieces(vid, tid, B, (2, 1, 1))
    cam = synth.orbit_cameras(13, 1, _dims(vol), 32, 24)[0]
    with pytest.raises(VrcError):
        R.render_piece(plan, 2, cam, (0, 0, 32, 24), 0.5, 1.0, B)  # no such piece
    with pytest.raises(VrcError):
        R.render_piece(plan, 0, cam, (20, 0, 20, 24), 0.5, 1.0, B)  # rect leaves the image
    with pytest.raises(VrcError):
        R.render_piece(plan, 0, cam, (0, 0, 32, 24), 0.5, 1.0, 16)  # brick size differs
    with pytest.raises(VrcError):
        R.render_sortlast(plan, cam, 0.5, 1.0, 0)
    with pytest.raises(VrcError):
        R.render_ordered(plan, cam, 0.5, 1.0, B, kernel=3)  # lane-group kernels
    a = torch.zeros((24, 32, 4), device="cuda")
    with pytest.raises(VrcError):
        R.composite([a, a], [(0, 0, 32, 24)] * 2, [0, 0], 32, 24)  # not a permutation
    R.update_tf(tid, tf, synth.CT_LO, synth.CT_HI)
    with pytest.raises(VrcError) as e:
        R.render_sortlast(plan, cam, 0.5, 1.0, B)  # the table changed since the plan
    assert "rebuild" in str(e.value)
    R.free_pieces(plan)
    with pytest.raises(VrcError):
        R.render_sortlast(plan, cam, 0.5, 1.0, B)
    R.free_volume(vid)
    R.free_tf(tid)


# ------------------------------------------------------------- full-size CT, sampled pixels

def test_full_size_pieces_match_oracle_on_sampled_pixels(R, orc, torch):
    # 512 x 512 x 400 CT at 1024^2, 2 x 2 x 2 pieces of 8^3 bricks: the blended image equals
    # the one-pass render to float32 rounding without termination (a property at any size),
    # and on 192 seeded pixels the sort-last and ordered images match the oracle's per-pixel
    # blend of its piece partials (sort-last) and its one-pass render (ordered), with
    # termination.
    vol = synth.ct_volume()
    dims = _dims(vol)
    B = 8
    vid, tid, tf = _scene(R, vol, B)
    plan = R.build_pieces(vid, tid, B, (2, 2, 2))
    pieces, _ = R.pieces(plan)
    cam = synth.orbit_cameras(4, 1, dims, 1024, 1024)[0]
    one = R.render(vid, tid, cam, 0.5, 1.0, B).cpu().numpy()
    sl = R.render_sortlast(plan, cam, 0.5, 1.0, B).cpu().numpy()
    assert np.abs(sl - one).max() <= 2e-5
    rng = np.random.default_rng(47)
    a = one[..., 3]
    cand = np.argwhere(a > 0.05)
    pix = [(int(x), int(y)) for y, x in cand[rng.choice(len(cand), 160, replace=False)]]
    pix += [(int(x), int(y)) for x, y in zip(rng.integers(0, 1024, 32), rng.integers(0, 1024, 32))]
    sl = R.render_sortlast(plan, cam, 0.5, 0.999, B).cpu().numpy()
    od = R.render_ordered(plan, cam, 0.5, 0.999, B).cpu().numpy()
    parts, flagged = [], np.zeros(len(pix), bool)
    for p in pieces:
        part, mg = orc.render_piece(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, B,
                                    p["brick_lo"], p["brick_hi"], ert=0.999, pixels=pix,
                                    return_margin=True)
        parts.append(part)
        flagged |= mg < ERT_MARGIN
    boxes = [(p["cell_lo"], p["cell_hi"]) for p in pieces]
    ref = orc.composite(np.stack(parts), orc.pixel_piece_order(cam, dims, boxes, pix))
    got = np.array([sl[y, x] for x, y in pix], np.float64)
    d = np.abs(got - ref).max(axis=-1)
    assert d[~flagged].max(initial=0.0) <= TOL and d[flagged].max(initial=0.0) <= 2e-3
    ref1, mg1 = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999, brick=B,
                           pixels=pix, return_margin=True)
    got1 = np.array([od[y, x] for x, y in pix], np.float64)
    d1 = np.abs(got1 - ref1).max(axis=-1)
    f1 = mg1 < ERT_MARGIN
    assert d1[~f1].max(initial=0.0) <= TOL and d1[f1].max(initial=0.0) <= 1e-3
    R.free_pieces(plan)
    R.free_volume(vid)
    R.free_tf(tid)
