"""GPU adjoint (vrc_render_backward, the torch.autograd wrapper) against the FP64 oracle's
reverse mode and against central finite differences of the FP64 forward (h = 1e-3).

Transfer-function gradients are continuous in the sample values and are compared entry by
entry (1e-3 relative). Voxel gradients jump where a sample's table coordinate crosses an
integer (the table is piecewise linear); float32 and float64 may place such a sample on
different sides, so a handful of voxels (< 0.1%) may differ by more than 1e-3 -- every other
significant voxel must agree to 1e-3, and all to 5e-2.
"""
import numpy as np
import pytest

from paper_2005_01442_gb300 import synth

pytestmark = pytest.mark.gpu


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


def _scene(seed=31, shape=(36, 40, 44)):
    vol = synth.ct_volume(shape, seed=seed).astype(np.float32)
    vol = vol + np.random.default_rng(seed).normal(0, 30, vol.shape).astype(np.float32)
    tf = synth.tf_ct(seed=4)
    return vol, tf


def _rel_check_tf(g, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    sig = np.abs(ref) > 1e-3 * scale
    err = np.abs(g - ref)
    assert np.all(err[sig] <= 1e-3 * np.abs(ref[sig]) + 1e-6 * scale), err[sig].max()
    assert np.all(err[~sig] <= 2e-6 * scale)


def _rel_check_vol(g, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    sig = np.abs(ref) > 1e-3 * scale
    err = np.abs(g - ref)
    ok = err <= 1e-3 * np.abs(ref) + 1e-6 * scale
    assert (~ok & sig).sum() <= max(1, int(1e-3 * sig.sum())), ((~ok & sig).sum(), sig.sum())
    assert np.all(err <= 5e-2 * scale)


@pytest.mark.parametrize("B", [0, 8])
@pytest.mark.parametrize("ert", [1.0, 0.999])
def test_backward_matches_oracle_reverse_mode(R, orc, torch, B, ert):
    vol, tf = _scene()
    lo, hi = synth.CT_LO, synth.CT_HI
    vid = R.upload_volume(vol)
    if B:
        R.build_bricks(vid, B)
    tid = R.set_tf(tf, lo, hi)
    rng = np.random.default_rng(5)
    for cam in synth.orbit_cameras(50, 2, synth.dims_of(vol), 40, 32):
        g = rng.normal(0, 1, (cam.height, cam.width, 4))
        if ert < 1.0:
            # pixels whose termination is decided within rounding carry no loss weight
            _, margin = orc.render(vol, tf, lo, hi, cam, 0.5, ert=ert, brick=B, return_margin=True)
            g[margin < 1e-5] = 0.0
        gt = torch.tensor(g, dtype=torch.float32, device="cuda")
        gtf = torch.zeros((256, 4), device="cuda")
        gvol = torch.zeros(vol.shape, device="cuda")
        R.render_backward(vid, tid, cam, gt, gtf, gvol, step=0.5, ert=ert, brick=B)
        rtf, rvol = orc.render_grad(vol, tf, lo, hi, cam, 0.5, g.astype(np.float32).astype(np.float64),
                                    ert=ert, brick=B)
        _rel_check_tf(gtf.cpu().numpy().astype(np.float64), rtf)
        _rel_check_vol(gvol.cpu().numpy().astype(np.float64), rvol)
    R.free_volume(vid)
    R.free_tf(tid)


def test_backward_same_with_and_without_leaping(R, torch):
    vol, tf = _scene(seed=33)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    R.build_bricks(vid, 16)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(51, 1, synth.dims_of(vol), 48, 40)[0]
    g = torch.randn((cam.height, cam.width, 4), device="cuda")
    out = {}
    for B in (0, 8, 16):
        gtf = torch.zeros((256, 4), device="cuda")
        gvol = torch.zeros(vol.shape, device="cuda")
        R.render_backward(vid, tid, cam, g, gtf, gvol, ert=0.999, brick=B)
        out[B] = (gtf, gvol)
    for B in (8, 16):
        for a, b in zip(out[B], out[0]):
            assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())
    R.free_volume(vid)


@pytest.mark.slow
def test_gradients_match_central_differences(R, orc, torch):
    """50 transfer-function entries and 50 voxels: GPU adjoint vs central differences of the
    FP64 forward (h = 1e-3 relative), skipping entries whose stencil straddles a kink."""
    vol, tf = _scene(seed=35, shape=(28, 32, 36))
    lo, hi = synth.CT_LO, synth.CT_HI
    tf = tf.copy()
    tf[:, 3] = np.maximum(tf[:, 3], 0.005)  # no opacity clamp kinks at a = 0
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    cams = synth.orbit_cameras(52, 2, synth.dims_of(vol), 24, 20)
    rng = np.random.default_rng(9)
    gs = [rng.normal(0, 1, (c.height, c.width, 4)).astype(np.float32) for c in cams]
    gtf = torch.zeros((256, 4), device="cuda")
    gvol = torch.zeros(vol.shape, device="cuda")
    for c, g in zip(cams, gs):
        R.render_backward(vid, tid, c, torch.tensor(g, device="cuda"), gtf, gvol, brick=8)
    gtf = gtf.cpu().numpy().astype(np.float64)
    gvol = gvol.cpu().numpy().astype(np.float64)

    def loss(v, t):
        return sum(float((orc.render(v, t, lo, hi, c, 0.5, brick=8) * g).sum())
                   for c, g in zip(cams, gs))

    checked = 0
    scale = np.abs(gtf).max()
    for flat in rng.permutation(np.flatnonzero(np.abs(gtf).ravel() > 1e-2 * scale)):
        k, ch = divmod(int(flat), 4)
        tp, tm = tf.astype(np.float64).copy(), tf.astype(np.float64).copy()
        h = 1e-3 * max(abs(float(tf[k, ch])), 1e-2)
        tp[k, ch] += h
        tm[k, ch] -= h
        tp32, tm32 = tp.astype(np.float32), tm.astype(np.float32)
        fd = (loss(vol, tp32) - loss(vol, tm32)) / (float(tp32[k, ch]) - float(tm32[k, ch]))
        assert abs(fd - gtf[k, ch]) <= 1e-3 * abs(gtf[k, ch]), (k, ch, fd, gtf[k, ch])
        checked += 1
        if checked == 50:
            break
    assert checked >= 20
    checked = 0
    vscale = np.abs(gvol).max()
    for vi in rng.permutation(np.flatnonzero(np.abs(gvol).ravel() > 0.05 * vscale)):
        def fd_at(hh):
            vp, vm = vol.copy(), vol.copy()
            vp.flat[vi] += hh
            vm.flat[vi] -= hh
            return (loss(vp, tf) - loss(vm, tf)) / (float(vp.flat[vi]) - float(vm.flat[vi]))
        hv = 1e-3 * max(1.0, abs(float(vol.flat[vi])))
        f1, f2 = fd_at(hv), fd_at(hv / 4)
        if abs(f1 - f2) > 1e-4 * abs(f1):
            continue  # kink of the piecewise-linear table inside the stencil
        assert abs(f1 - gvol.flat[vi]) <= 1e-3 * abs(gvol.flat[vi]), (vi, f1, gvol.flat[vi])
        checked += 1
        if checked == 50:
            break
    assert checked >= 20
    R.free_volume(vid)


def _pixel_weights(rng, cam, n):
    """A loss gradient that is zero except on n seeded pixels (N(0, 1) per channel)."""
    g = np.zeros((cam.height, cam.width, 4), np.float32)
    flat = rng.choice(cam.width * cam.height, size=n, replace=False)
    g.reshape(-1, 4)[flat] = rng.normal(0, 1, (n, 4)).astype(np.float32)
    return g, np.stack([flat % cam.width, flat // cam.width], -1)


@pytest.mark.slow
@pytest.mark.parametrize("forward", ["replay", "split"])
def test_backward_at_the_differentiation_config(R, orc, torch, forward):
    """The differentiation workload's own sizes: 256^3 float32 CT, 512^2 images, 8^3 bricks;
    4096 seeded pixels of each of 2 orbit cameras carry the loss. Gradients against the FP64
    oracle's reverse mode on the same pixels, with checkpoints rendered by the backward call
    itself (one ray per thread) or recorded by the split render."""
    vol = synth.ct_float_downsampled(7)
    tf = synth.tf_ct()
    lo, hi = synth.CT_LO, synth.CT_HI
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    rng = np.random.default_rng(14)
    gtf = torch.zeros((256, 4), device="cuda")
    gvol = torch.zeros(vol.shape, device="cuda")
    rtf = np.zeros((256, 4))
    rvol = np.zeros(vol.shape)
    for cam in synth.orbit_cameras(7, 2, synth.dims_of(vol), 512, 512):
        g, pix = _pixel_weights(rng, cam, 4096)
        gt = torch.tensor(g, device="cuda")
        ck = None
        if forward == "split":
            ck = R.ckpt_buffer(vid, cam, 0.5, 64)
            R.render(vid, tid, cam, brick=8, ckpt=ck)
        R.render_backward(vid, tid, cam, gt, gtf, gvol, step=0.5, brick=8, ckpt=ck)
        a, b = orc.render_grad(vol, tf, lo, hi, cam, 0.5, g.reshape(-1, 4)[pix[:, 1] * cam.width
                               + pix[:, 0]].astype(np.float64), brick=8, pixels=pix)
        rtf += a
        rvol += b
    _rel_check_tf(gtf.cpu().numpy().astype(np.float64), rtf)
    _rel_check_vol(gvol.cpu().numpy().astype(np.float64), rvol)
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("size", [1024, 1536])
def test_backward_at_image_sizes_with_fewer_lanes_per_ray(R, orc, torch, size):
    """Large images take fewer lanes per ray (4 at 1024^2, 2 at 1536^2): 2048 seeded pixels
    carry the loss (every other pixel has none and is skipped), checkpoints from the split
    render, gradients against the FP64 oracle's reverse mode on the same pixels."""
    vol, tf = _scene(seed=47, shape=(48, 56, 64))
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    rng = np.random.default_rng(48)
    cam = synth.orbit_cameras(49, 1, synth.dims_of(vol), size, size)[0]
    g, pix = _pixel_weights(rng, cam, 2048)
    ck = R.ckpt_buffer(vid, cam, 0.5, 64)
    R.render(vid, tid, cam, brick=8, ckpt=ck)
    gtf = torch.zeros((256, 4), device="cuda")
    gvol = torch.zeros(vol.shape, device="cuda")
    R.render_backward(vid, tid, cam, torch.tensor(g, device="cuda"), gtf, gvol, brick=8,
                      ckpt=ck)
    rtf, rvol = orc.render_grad(vol, tf, synth.CT_LO, synth.CT_HI, cam, 0.5,
                                g.reshape(-1, 4)[pix[:, 1] * cam.width + pix[:, 0]]
                                .astype(np.float64), brick=8, pixels=pix)
    _rel_check_tf(gtf.cpu().numpy().astype(np.float64), rtf)
    _rel_check_vol(gvol.cpu().numpy().astype(np.float64), rvol)
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("forward", ["replay", "ray", "split"])
def test_long_rays_with_hundreds_of_checkpoints(R, orc, torch, forward):
    """Rays of 6400 samples (a 48 x 48 x 1600 volume along z at step 0.25) in segments of 16:
    400 checkpoints per ray, compared with the FP64 oracle's reverse mode; a perspective view
    along the long axis as well."""
    vol = synth.ct_volume((1600, 48, 48), seed=41).astype(np.float32)
    tf = synth.tf_ct_dense()
    tf[:, 3] *= 0.1  # about 0.0012 opacity per voxel: rays cross the whole volume
    lo, hi = synth.CT_LO, synth.CT_HI
    dims = synth.dims_of(vol)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    cams = [synth.ortho_z_camera(dims, 12, 12),
            synth.Camera(0, (23.5, 27.0, -300.0), (23.5, 23.5, 800.0), (0.0, 1.0, 0.0), 4.0,
                         (0.0, 0.0), 10, 8).as_float32()]
    rng = np.random.default_rng(43)
    for cam in cams:
        g = rng.normal(0, 1, (cam.height, cam.width, 4)).astype(np.float32)
        gtf = torch.zeros((256, 4), device="cuda")
        gvol = torch.zeros(vol.shape, device="cuda")
        ck = None
        if forward != "replay":
            ck = R.ckpt_buffer(vid, cam, 0.25, 16)
            assert ck.numel() >= 400 * 4 * cam.width * cam.height
            R.render(vid, tid, cam, step=0.25, brick=8, ckpt=ck, seg_len=16,
                     kernel=1 if forward == "ray" else 0)
        R.render_backward(vid, tid, cam, torch.tensor(g, device="cuda"), gtf, gvol, step=0.25,
                          brick=8, seg_len=16, ckpt=ck)
        rtf, rvol = orc.render_grad(vol, tf, lo, hi, cam, 0.25, g.astype(np.float64), brick=8)
        _rel_check_tf(gtf.cpu().numpy().astype(np.float64), rtf)
        _rel_check_vol(gvol.cpu().numpy().astype(np.float64), rvol)
    R.free_volume(vid)
    R.free_tf(tid)


def test_recorded_checkpoints_equal_replayed_ones(R, torch):
    """Checkpoints recorded by the per-ray render equal the ones the backward renders itself
    (same kernel arithmetic), so the gradients agree up to the order of float atomics; the
    split render's checkpoints differ only by the rounding of its block compositing."""
    vol, tf = _scene(seed=39)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(54, 1, synth.dims_of(vol), 40, 36)[0]
    g = torch.randn((cam.height, cam.width, 4), device="cuda")
    out = {}
    for how in ("replay", "ray", "split"):
        gtf = torch.zeros((256, 4), device="cuda")
        gvol = torch.zeros(vol.shape, device="cuda")
        ck = None
        if how != "replay":
            ck = R.ckpt_buffer(vid, cam)
            R.render(vid, tid, cam, ert=0.999, brick=8, ckpt=ck, kernel=1 if how == "ray" else 6)
        R.render_backward(vid, tid, cam, g, gtf, gvol, ert=0.999, brick=8, ckpt=ck)
        out[how] = (gtf, gvol)
    for a, b in zip(out["ray"], out["replay"]):
        assert float((a - b).abs().max()) <= 1e-6 * float(b.abs().max())
    for a, b in zip(out["split"], out["replay"]):
        assert float((a - b).abs().max()) <= 2e-3 * float(b.abs().max())
    R.free_volume(vid)
    R.free_tf(tid)


@pytest.mark.parametrize("forward", ["replay", "split"])
def test_gradient_at_zero_opacity_from_above(R, orc, torch, forward):
    """grad_open_alpha: fully transparent table entries receive the gradient the oracle's
    derivative from above gives (brick 0: every sample carries gradient); with the default
    convention they receive none; with leaping the option is refused."""
    from paper_2005_01442_gb300 import native
    vol, _ = _scene(seed=44, shape=(28, 32, 36))
    tf = synth.tf_ct(seed=4)
    lo, hi = synth.CT_LO, synth.CT_HI
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, lo, hi)
    rng = np.random.default_rng(45)
    for cam in synth.orbit_cameras(56, 2, synth.dims_of(vol), 30, 24):
        g = rng.normal(0, 1, (cam.height, cam.width, 4)).astype(np.float32)
        gt = torch.tensor(g, device="cuda")
        ck = None
        if forward == "split":
            ck = R.ckpt_buffer(vid, cam)
            R.render(vid, tid, cam, brick=0, ckpt=ck)
        gtf = torch.zeros((256, 4), device="cuda")
        gvol = torch.zeros(vol.shape, device="cuda")
        R.render_backward(vid, tid, cam, gt, gtf, gvol, brick=0, ckpt=ck, open_alpha=True)
        rtf, rvol = orc.render_grad(vol, tf, lo, hi, cam, 0.5, g.astype(np.float64),
                                    open_alpha=True)
        zero = tf[:, 3] == 0.0
        assert np.abs(rtf[zero, 3]).max() > 0.0
        _rel_check_tf(gtf.cpu().numpy().astype(np.float64), rtf)
        _rel_check_vol(gvol.cpu().numpy().astype(np.float64), rvol)
        # entries inside a run of zero opacities: every sample that interpolates them has
        # opacity 0, so the default convention gives them no opacity gradient at all
        inner = zero.copy()
        inner[1:] &= zero[:-1]
        inner[:-1] &= zero[1:]
        assert np.abs(rtf[inner, 3]).max() > 0.0
        shut = torch.zeros((256, 4), device="cuda")
        R.render_backward(vid, tid, cam, gt, shut, None, brick=0, ckpt=ck)
        assert float(shut[torch.tensor(inner, device="cuda"), 3].abs().max()) == 0.0
        with pytest.raises(native.VrcError):
            R.render_backward(vid, tid, cam, gt, shut, None, brick=8, open_alpha=True)
    R.free_volume(vid)
    R.free_tf(tid)


def test_checkpoint_arguments_are_checked(R, torch):
    from paper_2005_01442_gb300 import native
    vol, tf = _scene(seed=40, shape=(20, 24, 28))
    vid = R.upload_volume(vol)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(55, 1, synth.dims_of(vol), 16, 12)[0]
    n = R.ckpt_bytes(vid, cam, 0.5, 64)
    K = -(-(int(np.ceil(np.sqrt(20 ** 2 + 24 ** 2 + 28 ** 2) / 0.5)) + 2) // 64)
    assert n >= 16 * 12 * (8 + 4 * K)
    ck = R.ckpt_buffer(vid, cam, 0.5, 24)
    with pytest.raises(native.VrcError):  # the split render checkpoints multiples of 16
        R.render(vid, tid, cam, ckpt=ck, seg_len=24, kernel=6)
    R.render(vid, tid, cam, ckpt=ck, seg_len=24, kernel=1)
    with pytest.raises(native.VrcError):  # lane-group kernels record no checkpoints
        R.render(vid, tid, cam, ckpt=ck, seg_len=24, kernel=3)
    with pytest.raises(native.VrcError):  # default variant only
        R.render(vid, tid, cam, ckpt=ck, seg_len=24, kernel=1, interp=1)
    with pytest.raises(native.VrcError):  # unaligned buffer
        R.render(vid, tid, cam, ckpt=ck[16:], seg_len=24, kernel=1)
    R.free_volume(vid)
    R.free_tf(tid)


def test_autograd_function(R, torch):
    from paper_2005_01442_gb300.autograd import DifferentiableRenderer
    vol, tf = _scene(seed=37, shape=(32, 36, 40))
    dr = DifferentiableRenderer(R, vol.shape, synth.CT_LO, synth.CT_HI)
    v = torch.tensor(vol, device="cuda", requires_grad=True)
    t = torch.tensor(tf, requires_grad=True)
    cams = synth.orbit_cameras(53, 2, synth.dims_of(vol), 32, 24)
    target = torch.rand((24, 32, 4), device="cuda")
    loss = sum(((dr(v, t, c, brick=8, ert=0.999) - target) ** 2).sum() for c in cams)
    loss.backward()
    # same gradients straight through the C ABI
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(tf, synth.CT_LO, synth.CT_HI)
    gtf = torch.zeros((256, 4), device="cuda")
    gvol = torch.zeros(vol.shape, device="cuda")
    for c in cams:  # the autograd forward records checkpoints with the split render
        ck = R.ckpt_buffer(vid, c)
        img = R.render(vid, tid, c, brick=8, ert=0.999, ckpt=ck)
        R.render_backward(vid, tid, c, 2 * (img - target), gtf, gvol, brick=8, ert=0.999,
                          ckpt=ck)
    assert float((t.grad.cuda() - gtf).abs().max()) <= 1e-5 * float(gtf.abs().max())
    assert float((v.grad - gvol).abs().max()) <= 1e-5 * float(gvol.abs().max())
    R.free_volume(vid)
