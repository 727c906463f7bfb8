"""GPU parity of libvrc against the FP64 oracle, through the C ABI.

Tolerances: images within max |d| <= 1e-4 per RGBA channel of the oracle; brick tables and
occupancy bytes bit-exact; empty-space leaping bit-identical to no leaping. Where early ray
termination is on, a pixel whose opacity passes the threshold within 1e-5 of it may stop one
sample apart in float32 and float64; such pixels (flagged by the oracle's margin) are held to
the termination bound 1e-3 instead.
"""
import numpy as np
import pytest

from paper_2005_01442_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
ERT_MARGIN = 1e-5
ERT_BOUND = 1e-3


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


def _check(img, ref, margin=None, tol=TOL):
    img = np.asarray(img, np.float64).reshape(ref.shape)
    d = np.abs(img - ref).max(axis=-1)
    if margin is not None:
        flagged = margin.reshape(d.shape) < ERT_MARGIN
        assert d[~flagged].max(initial=0.0) <= tol, d[~flagged].max(initial=0.0)
        assert d[flagged].max(initial=0.0) <= ERT_BOUND
        return d, flagged
    assert d.max() <= tol, (d.max(), np.unravel_index(d.argmax(), d.shape))
    return d, None


def _ct_small(seed=21, shape=(48, 64, 72)):
    return synth.ct_volume(shape, seed=seed)


# ------------------------------------------------------------------- a1, a2: exact tables

@pytest.mark.parametrize("kind", ["u16", "i16", "f32"])
@pytest.mark.parametrize("B", [8, 16])
def test_brick_tables_bit_exact(R, orc, kind, B):
    if kind == "u16":
        vol = synth.phantom(40, seed=3)[:, :37, :]
    elif kind == "i16":
        vol = _ct_small(shape=(45, 50, 61))
    else:
        vol = np.random.default_rng(4).normal(0, 50, (33, 29, 47)).astype(np.float32)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, B)
    mn, mx = R.bricks(vid, B)
    rmn, rmx = orc.bricks(vol, B)
    assert mn.dtype == rmn.dtype and np.array_equal(mn, rmn) and np.array_equal(mx, rmx)
    R.free_volume(vid)


@pytest.mark.parametrize("B", [8, 16])
def test_occupancy_bit_exact(R, orc, B):
    vol = _ct_small()
    vid = R.upload_volume(vol)
    R.build_bricks(vid, B)
    for seed in (None, 1, 2):
        tf = synth.tf_ct(seed)
        tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
        occ = R.occupancy(vid, tid, B)
        ref = orc.occupancy(*orc.bricks(vol, B), tf, synth.CT_LO, synth.CT_HI)
        assert np.array_equal(occ, ref)
        R.free_tf(tid)
    R.free_volume(vid)


# ------------------------------------------------------------- a3-a9: images vs the oracle

@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
def test_phantom_orthographic_parity(R, orc, torch, kernel):
    """64^3 uint16 phantom, 128^2 orthographic along +z, step 0.5, no skipping."""
    vol = synth.phantom()
    tf = synth.tf_random(2)
    cam = synth.ortho_z_camera((64, 64, 64), 128, 128)
    vid = R.upload_volume(vol)
    tid = R.set_tf(tf, synth.PHANTOM_LO, synth.PHANTOM_HI)
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    img = R.render(vid, tid, cam, step=0.5, counters=cnt, kernel=kernel).cpu().numpy()
    ref = orc.render(vol, tf, synth.PHANTOM_LO, synth.PHANTOM_HI, cam, 0.5)
    _check(img, ref)
    assert cnt.tolist() == [2097152, 2097152, 2097152]  # no skipping: all resampled
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("B", [0, 8, 16])
@pytest.mark.parametrize("ert", [1.0, 0.999])
def test_ct_perspective_parity(R, orc, torch, B, ert, kernel):
    vol = _ct_small()
    tf = synth.tf_ct()
    vid = R.upload_volume(vol)
    if B:
        R.build_bricks(vid, B)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(40, 3, synth.dims_of(vol), 96, 80):
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        img = R.render(vid, tid, cam, step=0.5, ert=ert, brick=B, counters=cnt,
                       kernel=kernel).cpu().numpy()
        ref, margin, rc = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=ert,
                                     brick=B, return_margin=True, return_counts=True)
        _check(img, ref, margin if ert < 1 else None)
        assert cnt[0].item() == rc[0] or abs(cnt[0].item() - rc[0]) <= 8  # segment counts
        # executed: samples in occupied bricks up to termination, as the oracle counts them
        # (a pixel whose termination float rounding decides may stop one sample apart)
        assert cnt[2].item() <= cnt[1].item()  # resampled: executed minus clear cells
        if B == 0:
            assert cnt[2].item() == cnt[1].item()
        if ert >= 1.0:
            assert cnt[1].item() == rc[1]
        else:
            assert abs(cnt[1].item() - rc[1]) <= int((margin < ERT_MARGIN).sum()) + 8
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
def test_empty_space_leaping_bit_identical(R, torch, kernel):
    """Skipping (leaps over empty bricks, clear cells) changes no pixel, bit for bit."""
    vol = _ct_small(seed=5)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    R.build_bricks(vid, 16)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(41, 4, synth.dims_of(vol), 120, 90):
        for ert in (1.0, 0.999):
            c0 = torch.zeros(3, dtype=torch.int64, device="cuda")
            ref = R.render(vid, tid, cam, ert=ert, brick=0, counters=c0, kernel=kernel)
            for B in (8, 16):
                c1 = torch.zeros(3, dtype=torch.int64, device="cuda")
                img = R.render(vid, tid, cam, ert=ert, brick=B, counters=c1, kernel=kernel)
                assert torch.equal(img, ref)
                assert c1[0] == c0[0] and c1[1] < c0[1]
    R.free_volume(vid)


def test_early_termination_bound(R, torch):
    vol = _ct_small(seed=6)
    tf = synth.tf_ct().copy()
    tf[:, 3] = np.minimum(tf[:, 3] * 3.0, 0.95)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(42, 2, synth.dims_of(vol), 96, 80):
        full = R.render(vid, tid, cam, ert=1.0, brick=8).cpu().numpy().astype(np.float64)
        ert = R.render(vid, tid, cam, ert=0.999, brick=8).cpu().numpy().astype(np.float64)
        stopped = ert[..., 3] > 0.999
        assert stopped.any()
        d = np.abs(full - ert).max(-1)
        assert np.all(d[stopped] <= (1.0 - ert[..., 3])[stopped] + 1e-6)
    R.free_volume(vid)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
def test_float_volume_and_ragged_sizes(R, orc, kernel):
    rng = np.random.default_rng(9)
    vol = (rng.normal(0, 1, (13, 17, 19)).cumsum(0) * 40).astype(np.float32)
    tf = synth.tf_random(7, 5)
    tf[:, 3] *= 0.4
    lo, hi = float(vol.min()), float(vol.max())
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    dims = synth.dims_of(vol)
    for cam in synth.orbit_cameras(43, 2, dims, 37, 23) + [synth.ortho_z_camera(dims, 29, 31)]:
        for B in (0, 8):
            img = R.render(vid, tid, cam, step=0.37, brick=B, kernel=kernel).cpu().numpy()
            ref = orc.render(vol, tf, lo, hi, cam, 0.37, brick=B)
            _check(img, ref)
    R.free_volume(vid)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
def test_degenerate_cases(R, orc, kernel):
    tf = synth.tf_random(3)
    # 1x1x1 volume, 1x1 image, step longer than the box
    vol = np.array([[[1234]]], np.uint16)
    vid = R.upload_volume(vol)
    tid = R.set_tf(tf, 0, 4095)
    cam = synth.ortho_z_camera((1, 1, 1), 1, 1)
    img = R.render(vid, tid, cam, step=3.0, kernel=kernel).cpu().numpy()
    _check(img, orc.render(vol, tf, 0, 4095, cam, 3.0))
    # camera looking away from the volume: every ray misses, black transparent image
    vol = synth.phantom(16)
    vid2 = R.upload_volume(vol)
    away = synth.Camera(0, (7.5, 7.5, -20.0), (7.5, 7.5, -40.0), (0, 1, 0), 30.0, (0, 0), 8, 8)
    assert np.all(R.render(vid2, tid, away, kernel=kernel).cpu().numpy() == 0.0)
    # eye inside the volume
    inside = synth.Camera(0, (7.3, 8.1, 6.6), (0.0, 3.0, 15.0), (0, 1, 0), 60.0, (0, 0), 16, 12)
    img = R.render(vid2, tid, inside, step=0.25, kernel=kernel).cpu().numpy()
    _check(img, orc.render(vol, tf, 0, 4095, inside, 0.25))
    R.free_volume(vid)
    R.free_volume(vid2)


def test_invalid_arguments_are_rejected(R, torch):
    from paper_2005_01442_gb300.native import VrcError
    vol = synth.phantom(16)
    vid = R.upload_volume(vol)
    tid = R.set_tf(synth.tf_random(3), 0, 4095)
    cam = synth.ortho_z_camera((16, 16, 16), 8, 8)
    with pytest.raises(VrcError, match="VRC_ERR_ARG"):
        R.render(vid + 1000, tid, cam)
    with pytest.raises(VrcError, match="VRC_ERR_ARG"):
        R.render(vid, tid, cam, step=0.0)
    with pytest.raises(VrcError, match="VRC_ERR_ARG"):
        R.render(vid, tid, cam, brick=4)
    with pytest.raises(VrcError, match="VRC_ERR_STATE"):
        R.render(vid, tid, cam, brick=8)  # no brick table yet
    with pytest.raises(VrcError, match="VRC_ERR_ARG"):
        R.set_tf(synth.tf_random(3), 5.0, 5.0)
    bad = synth.Camera(0, (1, 2, 3), (1, 2, 3), (0, 1, 0), 30.0, (0, 0), 8, 8)
    with pytest.raises(VrcError, match="VRC_ERR_ARG"):
        R.render(vid, tid, bad)
    assert R.last_device_error() == 0
    R.free_volume(vid)


def test_render_host_matches_device(R, torch):
    vol = _ct_small(seed=8)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 16)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(44, 1, synth.dims_of(vol), 64, 48)[0]
    dev = R.render(vid, tid, cam, ert=0.999, brick=16).cpu()
    host = R.render_host(vid, tid, cam, ert=0.999, brick=16)
    assert torch.equal(dev, host)
    R.free_volume(vid)


@pytest.mark.parametrize("kernel", [0, 1])
def test_render_host_batch_matches_device(R, torch, kernel):
    # double-buffered read-back: every frame equals its device render bit for bit, for mixed
    # image sizes (the buffers grow mid-way), one camera, and no camera
    import numpy as np
    vol = _ct_small(seed=9)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    dims = synth.dims_of(vol)
    cams = (list(synth.orbit_cameras(45, 3, dims, 40, 32)) + list(synth.orbit_cameras(46, 2, dims, 72, 56))
            + [synth.ortho_z_camera(dims, 33, 17)])
    outs = R.render_host_batch(vid, tid, cams, ert=0.999, brick=8, kernel=kernel)
    for c, h in zip(cams, outs):
        assert torch.equal(R.render(vid, tid, c, ert=0.999, brick=8, kernel=kernel).cpu(), h)
    one = [np.zeros((cams[0].height, cams[0].width, 4), np.float32)]
    R.render_host_batch(vid, tid, cams[:1], out=one, ert=0.999, brick=8, kernel=kernel)
    assert np.array_equal(one[0], R.render(vid, tid, cams[0], ert=0.999, brick=8,
                                           kernel=kernel).cpu().numpy())
    assert R.render_host_batch(vid, tid, [], ert=0.999, brick=8) == []
    R.free_volume(vid)


# --------------------------------------------------------- full-size CT, sampled pixels

@pytest.fixture(scope="module")
def ct_full(R):
    vol = synth.ct_volume()  # 512 x 512 x 400 int16
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    R.build_bricks(vid, 16)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    yield vol, vid, tid
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("B", [8, 16])
def test_ct_full_size_sampled_parity(R, orc, torch, ct_full, B, kernel):
    """512^2 x 400 CT, 1024^2 perspective, step 0.5, ESL, ERT 0.999: 4096 sampled pixels per
    camera against the oracle; ESL bit-identical to no ESL on the whole image."""
    vol, vid, tid = ct_full
    tf = synth.tf_ct()
    rng = np.random.default_rng(B)
    for cam in synth.orbit_cameras(4, 2, synth.dims_of(vol), 1024, 1024):
        img = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=B, kernel=kernel).cpu().numpy()
        pix = np.stack([rng.integers(0, 1024, 4096), rng.integers(0, 1024, 4096)], -1)
        ref, margin = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999,
                                 brick=B, pixels=pix, return_margin=True)
        _check(img[pix[:, 1], pix[:, 0]], ref, margin)
        noesl = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=0, kernel=kernel).cpu().numpy()
        assert np.array_equal(img, noesl)


@pytest.mark.parametrize("tf_kind", ["ct", "dense"])
def test_tma_staged_render_equals_per_ray_kernel(R, torch, ct_full, tf_kind):
    """The TMA-staged render (kernel 7) resamples from shared memory in the per-ray kernel's
    order: the same image bit for bit, and the same sample counts, on the full-size CT with
    both transfer functions, 1024^2 and 256^2 images (the latter covering several voxels per
    pixel, where some windows fall back to L1)."""
    vol, vid, tid = ct_full
    if tf_kind == "dense":
        tid = R.set_tf(synth.tf_ct_dense(), synth.CT_LO, synth.CT_HI)
    for size in (1024, 256):
        for cam in synth.orbit_cameras(11, 2, synth.dims_of(vol), size, size):
            for B in (0, 8):
                ca = torch.zeros(3, dtype=torch.int64, device="cuda")
                cb = torch.zeros(3, dtype=torch.int64, device="cuda")
                a = R.render(vid, tid, cam, ert=0.999, brick=B, kernel=1, counters=ca)
                b = R.render(vid, tid, cam, ert=0.999, brick=B, kernel=7, counters=cb)
                assert torch.equal(a, b), (size, B, float((a - b).abs().max()))
                assert torch.equal(ca, cb)
    if tf_kind == "dense":
        R.free_tf(tid)
    assert R.last_device_error() == 0


def test_dense_tf_full_size_sampled_parity(R, orc, torch, ct_full):
    """The dense transfer function (long rays, nearly every sample resampled) on the full-size
    CT at 1024^2: 2048 sampled pixels of the split render and of the TMA-staged render against
    the oracle."""
    vol, vid, _ = ct_full
    tf = synth.tf_ct_dense()
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    rng = np.random.default_rng(12)
    cam = synth.orbit_cameras(13, 1, synth.dims_of(vol), 1024, 1024)[0]
    pix = np.stack([rng.integers(0, 1024, 2048), rng.integers(0, 1024, 2048)], -1)
    ref, margin = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999, brick=8,
                             pixels=pix, return_margin=True)
    for kernel in (0, 7):
        img = R.render(vid, tid, cam, ert=0.999, brick=8, kernel=kernel).cpu().numpy()
        _check(img[pix[:, 1], pix[:, 0]], ref, margin)
    R.free_tf(tid)


def test_kernels_agree(R, torch, ct_full):
    """The per-ray and the lane-group kernels compute the same image up to float rounding of
    the compositing order."""
    vol, vid, tid = ct_full
    for cam in synth.orbit_cameras(7, 2, synth.dims_of(vol), 512, 512):
        a = R.render(vid, tid, cam, ert=0.999, brick=8, kernel=1)
        for k in (2, 3, 4, 5, 6):
            b = R.render(vid, tid, cam, ert=0.999, brick=8, kernel=k)
            d = (a - b).abs()
            # pixels whose termination is decided within float rounding may differ by <= 1e-3
            assert float(d.max()) <= 1e-3, k
            assert float((d > 1e-5).float().mean()) < 1e-3, k


# ------------------------------------------- split render: the second phase and its queue

def _glass_tf(alpha):
    """Every value has the same small opacity: rays never terminate early and every sample
    has non-zero opacity, so every ray longer than the hand-over point is queued."""
    tf = np.zeros((256, 4), np.float32)
    tf[:, 0] = np.linspace(0.2, 1.0, 256)
    tf[:, 1] = np.linspace(1.0, 0.3, 256)
    tf[:, 2] = 0.5
    tf[:, 3] = alpha
    return tf


@pytest.mark.parametrize("B", [0, 8])
def test_split_long_rays_parity_and_sample_count(R, orc, torch, B):
    """All rays long: phase two renders nearly every pixel. Images match the oracle and the
    sample counter shows every sample composited exactly once across the two phases."""
    vol = _ct_small(seed=5, shape=(40, 44, 36))
    tf = _glass_tf(0.02)
    vid = R.upload_volume(vol)
    if B:
        R.build_bricks(vid, B)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in (synth.ortho_z_camera(synth.dims_of(vol), 37, 29),
                synth.orbit_cameras(9, 1, synth.dims_of(vol), 45, 38)[0]):
        ref, (onom, _) = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=1.0,
                                    return_counts=True)
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        img = R.render(vid, tid, cam, step=0.5, ert=1.0, brick=B, counters=cnt, kernel=6)
        _check(img.cpu().numpy(), ref)
        nominal, executed, resampled = cnt.tolist()
        assert nominal == onom and resampled <= executed
        if B == 0:
            assert executed == nominal == resampled
        one = R.render(vid, tid, cam, step=0.5, ert=1.0, brick=B, kernel=1)
        assert float((img - one).abs().max()) <= 1e-5
    R.free_tf(tid)
    R.free_volume(vid)


def test_split_queue_grows_and_streams_are_independent(R, torch):
    """A larger image grows the queue; renders on two streams use separate queues and give
    the same images as on the default stream."""
    vol = _ct_small(seed=6)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(_glass_tf(0.01), synth.CT_LO, synth.CT_HI)
    cams = [synth.orbit_cameras(11, 1, synth.dims_of(vol), w, h)[0]
            for w, h in ((24, 16), (96, 80), (130, 70))]
    ref = [R.render(vid, tid, c, ert=0.999, brick=8, kernel=6).clone() for c in cams]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for k in range(3):
        for i, c in enumerate(cams):
            outs.append((i, R.render(vid, tid, c, ert=0.999, brick=8, kernel=6,
                                     stream=s1 if (i + k) % 2 else s2)))
    torch.cuda.synchronize()
    for i, img in outs:
        assert torch.equal(img, ref[i])
    R.free_tf(tid)
    R.free_volume(vid)


# ------------------------------------------------------- cell transparency mask (a10)

@pytest.mark.parametrize("kind", ["u16", "i16", "f32"])
def test_cell_mask_bit_exact(R, orc, kind):
    """The GPU cell mask equals the oracle's byte for byte (ragged sizes across word
    boundaries; every dtype)."""
    if kind == "u16":
        vol = synth.phantom(40, seed=3)[:, :37, :]
        tf, lo, hi = synth.tf_random(5).copy(), synth.PHANTOM_LO, synth.PHANTOM_HI
        tf[:120, 3] = 0.0  # a transparent low range
    elif kind == "i16":
        vol = _ct_small(shape=(45, 50, 63))
        tf, lo, hi = synth.tf_ct(), synth.CT_LO, synth.CT_HI
    else:
        vol = (np.random.default_rng(4).normal(0, 1, (33, 29, 70)).cumsum(0) * 60).astype(
            np.float32)
        tf, lo, hi = synth.tf_random(8, 5).copy(), -300.0, 300.0
        tf[:200, 3] = 0.0
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    got = R.cellmask(vid, tid, 8)
    ref = orc.cellmask(vol, tf, lo, hi)
    assert 0 < ref.sum() < ref.size
    assert np.array_equal(got, ref)
    R.free_tf(tid)
    R.free_volume(vid)


def test_cell_mask_follows_updates(R, orc):
    """The mask is rebuilt when the volume or the table changes."""
    vol = _ct_small(seed=8)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tf = synth.tf_ct()
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    assert np.array_equal(R.cellmask(vid, tid, 8), orc.cellmask(vol, tf, synth.CT_LO, synth.CT_HI))
    tf2 = synth.tf_ct(3)
    R.update_tf(tid, tf2, synth.CT_LO, synth.CT_HI)
    assert np.array_equal(R.cellmask(vid, tid, 8),
                          orc.cellmask(vol, tf2, synth.CT_LO, synth.CT_HI))
    vol2 = vol.copy()
    vol2[10:20, 5:30, 7:40] = 1300
    R.update_volume(vid, vol2)
    R.build_bricks(vid, 8)
    assert np.array_equal(R.cellmask(vid, tid, 8),
                          orc.cellmask(vol2, tf2, synth.CT_LO, synth.CT_HI))
    R.free_tf(tid)
    R.free_volume(vid)


@pytest.mark.parametrize("pattern", ["alternate", "all_zero", "all_open", "blocks"])
def test_cell_mask_zero_runs(R, orc, pattern):
    """Tables with many, one or no runs of zero opacity (the mask kernel reduces taps to the
    id of the zero run holding them): still equal to the oracle's min/max rule."""
    vol = _ct_small(seed=11, shape=(37, 41, 70))
    tf = synth.tf_ct().copy()
    if pattern == "alternate":
        tf[:, 3] = np.where(np.arange(256) % 2 == 1, 0.2, 0.0)
    elif pattern == "all_zero":
        tf[:, 3] = 0.0
    elif pattern == "all_open":
        tf[:, 3] = 0.05
    else:
        tf[:, 3] = np.where((np.arange(256) // 7) % 3 == 0, 0.3, 0.0)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    got = R.cellmask(vid, tid, 8)
    ref = orc.cellmask(vol, tf, synth.CT_LO, synth.CT_HI)
    assert np.array_equal(got, ref)
    if pattern == "all_zero":
        assert ref.sum() == 0
    if pattern == "all_open":
        assert ref.all()
    R.free_tf(tid)
    R.free_volume(vid)


# ------------------------------- interpolation / classification variants (the next row 1)

VARIANTS = [(1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("interp,preclass", VARIANTS)
@pytest.mark.parametrize("kernel", [0, 1, 6])
@pytest.mark.parametrize("B", [0, 8])
def test_variant_parity(R, orc, torch, interp, preclass, kernel, B):
    """Trilinear and pre-classification variants against the oracle (perspective CT views,
    ERT 0.999), and skipping bit-identical to no skipping."""
    vol = _ct_small(seed=15, shape=(44, 52, 60))
    tf = synth.tf_ct(2)
    vid = R.upload_volume(vol)
    if B:
        R.build_bricks(vid, B)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(43, 2, synth.dims_of(vol), 72, 60):
        img = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=B, kernel=kernel,
                       interp=interp, preclass=preclass).cpu().numpy()
        ref, margin = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999,
                                 brick=B, return_margin=True, interp=interp, preclass=preclass)
        _check(img, ref, margin)
        if B:
            noesl = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=0, kernel=kernel,
                             interp=interp, preclass=preclass).cpu().numpy()
            assert np.array_equal(img, noesl)
    R.free_tf(tid)
    R.free_volume(vid)


def test_variants_change_the_image_and_are_rejected_where_unsupported(R, torch):
    vol = _ct_small(seed=16)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(44, 1, synth.dims_of(vol), 64, 64)[0]
    base = R.render(vid, tid, cam, ert=0.999, brick=8)
    for interp, preclass in VARIANTS:
        img = R.render(vid, tid, cam, ert=0.999, brick=8, interp=interp, preclass=preclass)
        assert float((img - base).abs().max()) > 1e-3
    from paper_2005_01442_gb300 import native
    for kernel in (2, 3, 4, 5):
        with pytest.raises(native.VrcError):
            R.render(vid, tid, cam, ert=0.999, brick=8, kernel=kernel, interp=1)
    with pytest.raises(native.VrcError):
        R.render(vid, tid, cam, interp=2)
    R.free_tf(tid)
    R.free_volume(vid)


def test_variants_rejected_by_adjoint_and_server(R, torch):
    import ctypes as C
    from paper_2005_01442_gb300 import native
    vol = _ct_small(seed=17).astype(np.float32)
    vid = R.upload_volume(vol)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(45, 1, synth.dims_of(vol), 16, 16)[0]
    g = torch.zeros((16, 16, 4), device="cuda")
    gtf = torch.zeros((256, 4), device="cuda")
    st = R.lib.vrc_render_backward(R.ctx, vid, tid, C.byref(native.camera_struct(cam)),
                                   C.byref(native.params_struct(0.5, 1.0, 0, 64, 0, 1, 0)),
                                   C.c_void_p(g.data_ptr()), None, C.c_void_p(gtf.data_ptr()),
                                   None, None)
    assert st == -1
    srv = C.c_void_p()
    native.check(R.ctx, R.lib.vrc_server_create(R.ctx, 4, C.byref(srv)))
    out = torch.empty((16, 16, 4), device="cuda")
    t = C.c_longlong()
    st = R.lib.vrc_server_submit(srv, vid, tid, C.byref(native.camera_struct(cam)),
                                 C.byref(native.params_struct(0.5, 1.0, 0, 64, 0, 0, 1)),
                                 C.c_void_p(out.data_ptr()), C.byref(t))
    assert st == -1
    R.lib.vrc_server_destroy(srv)
    R.free_tf(tid)
    R.free_volume(vid)


# --------------------------------------------------- local lighting (the next row 2)

PHONG = (0.3, 0.7, 0.25, 16.0)


@pytest.mark.parametrize("kernel", [0, 1, 6])
@pytest.mark.parametrize("B", [0, 8])
def test_phong_parity(R, orc, torch, kernel, B):
    """Headlight Blinn-Phong from the B-spline gradient against the oracle; skipping
    bit-identical to no skipping; opacity equal to the unshaded render."""
    vol = _ct_small(seed=18, shape=(44, 52, 60))
    tf = synth.tf_ct(1)
    vid = R.upload_volume(vol)
    if B:
        R.build_bricks(vid, B)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(46, 2, synth.dims_of(vol), 72, 60):
        img = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=B, kernel=kernel,
                       phong=PHONG).cpu().numpy()
        ref, margin = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5, ert=0.999,
                                 brick=B, return_margin=True, phong=PHONG)
        _check(img, ref, margin)
        plain = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=B, kernel=kernel)
        assert np.array_equal(img[..., 3], plain.cpu().numpy()[..., 3])
        if B:
            noesl = R.render(vid, tid, cam, step=0.5, ert=0.999, brick=0, kernel=kernel,
                             phong=PHONG).cpu().numpy()
            assert np.array_equal(img, noesl)
    R.free_tf(tid)
    R.free_volume(vid)


def test_phong_argument_checks(R, torch):
    from paper_2005_01442_gb300 import native
    vol = _ct_small(seed=19)
    vid = R.upload_volume(vol)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(47, 1, synth.dims_of(vol), 16, 16)[0]
    bad = [dict(phong=PHONG, interp=1), dict(phong=PHONG, preclass=1),
           dict(phong=(0.3, 0.7, 0.2, 0.0)), dict(phong=(-0.1, 0.7, 0.2, 8.0)),
           dict(phong=PHONG, kernel=3)]
    for kw in bad:
        with pytest.raises(native.VrcError):
            R.render(vid, tid, cam, **kw)
    R.free_tf(tid)
    R.free_volume(vid)


# ------------------------------------- pre-integrated classification (the next row 3)

@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("step,ert", [(0.5, 0.999), (0.37, 1.0)])
def test_preint_parity(R, orc, torch, kernel, step, ert):
    """Slabs through the pre-integration table against the oracle (table built on the GPU
    in double, looked up bilinearly in float)."""
    vol = _ct_small(seed=20, shape=(40, 48, 56))
    tf = synth.tf_ct(3)
    vid = R.upload_volume(vol)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    for cam in synth.orbit_cameras(48, 2, synth.dims_of(vol), 64, 56):
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        img = R.render(vid, tid, cam, step=step, ert=ert, kernel=kernel, preint=1,
                       counters=cnt).cpu().numpy()
        ref, margin, (nom, ex) = orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, step,
                                            ert=ert, return_margin=True, return_counts=True,
                                            preint=1)
        _check(img, ref, margin if ert < 1 else None)
        if ert >= 1.0:
            assert cnt.tolist() == [nom, ex, ex]
    R.free_tf(tid)
    R.free_volume(vid)


def test_preint_table_follows_step_and_table_and_rejects(R, orc, torch):
    from paper_2005_01442_gb300 import native
    vol = _ct_small(seed=21, shape=(30, 34, 38))
    tf = synth.tf_ct()
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(49, 1, synth.dims_of(vol), 40, 40)[0]
    for step in (0.5, 0.3, 0.5):
        img = R.render(vid, tid, cam, step=step, preint=1).cpu().numpy()
        _check(img, orc.render(vol, tf, synth.CT_LO, synth.CT_HI, cam, step, preint=1))
    tf2 = synth.tf_ct(4)
    R.update_tf(tid, tf2, synth.CT_LO, synth.CT_HI)
    img = R.render(vid, tid, cam, step=0.5, preint=1).cpu().numpy()
    _check(img, orc.render(vol, tf2, synth.CT_LO, synth.CT_HI, cam, 0.5, preint=1))
    for kw in (dict(brick=8), dict(interp=1), dict(phong=(0.3, 0.7, 0.2, 8.0)), dict(kernel=6),
               dict(kernel=2)):
        with pytest.raises(native.VrcError):
            R.render(vid, tid, cam, preint=1, **kw)
    R.free_tf(tid)
    R.free_volume(vid)
