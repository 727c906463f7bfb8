"""vrc_render_noalloc: the render entry point for callers that must not allocate device memory
while rendering (a fixed, pre-reserved memory budget, or no tolerance for the device-wide
synchronisation of cudaMalloc/cudaFree). It keeps its occupancy and leaping fields in one
fixed device array instead of context allocations; its images must equal vrc_render's.

This file is collected last on purpose: it only adds a second path to an existing one.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2005_01442_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_01442_gb300 import build, native
    from paper_2005_01442_gb300.renderer import Renderer
    build.build()
    R = Renderer(0)
    yield torch, native, R
    R.close()


def _noalloc(torch, native, R, vid, tid, cam, B, kernel, out, cnt):
    st = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    return R.lib.vrc_render_noalloc(R.ctx, vid, tid, C.byref(native.camera_struct(cam)),
                                    C.byref(native.params_struct(0.5, 0.999, B, 64, kernel)),
                                    C.c_void_p(out.data_ptr()),
                                    C.c_void_p(cnt.data_ptr()) if cnt is not None else None, st)


def test_noalloc_render_matches_render(env):
    torch, native, R = env
    vol = synth.ct_volume((96, 112, 128), seed=13)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    R.build_bricks(vid, 16)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cams = synth.orbit_cameras(23, 2, synth.dims_of(vol), 160, 128)
    for B in (8, 16):
        for kernel in (1, 2):
            for cam in cams:  # two calls in a row share (and overwrite) the fixed array
                c0 = torch.zeros(3, dtype=torch.int64, device="cuda")
                ref = R.render(vid, tid, cam, ert=0.999, brick=B, kernel=kernel, counters=c0)
                out = torch.full_like(ref, float("nan"))
                c1 = torch.zeros(3, dtype=torch.int64, device="cuda")
                native.check(R.ctx, _noalloc(torch, native, R, vid, tid, cam, B, kernel, out, c1))
                torch.cuda.synchronize()
                assert float((out - ref).abs().max()) <= 1e-4
                assert torch.equal(out, ref) and torch.equal(c0, c1)
    assert R.last_device_error() == 0
    R.free_volume(vid)
    R.free_tf(tid)


def test_noalloc_render_without_room_for_the_cell_mask(env):
    """A volume whose cell-mask build scratch does not fit behind the brick fields (256 x 256 x
    128: about 9 MB of run ids) renders without clear-cell skipping: the same pixels as
    vrc_render, bit for bit, and at least as many executed samples."""
    torch, native, R = env
    vol = synth.ct_volume((128, 256, 256), seed=15)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    R.build_bricks(vid, 16)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cams = synth.orbit_cameras(25, 2, synth.dims_of(vol), 96, 80)
    for B in (8, 16):
        for cam in cams:  # two calls in a row
            c0 = torch.zeros(3, dtype=torch.int64, device="cuda")
            ref = R.render(vid, tid, cam, ert=0.999, brick=B, kernel=1, counters=c0)
            out = torch.full_like(ref, float("nan"))
            c1 = torch.zeros(3, dtype=torch.int64, device="cuda")
            native.check(R.ctx, _noalloc(torch, native, R, vid, tid, cam, B, 1, out, c1))
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
            assert int(c1[0]) == int(c0[0]) and int(c1[1]) >= int(c0[1])
    assert R.last_device_error() == 0
    R.free_volume(vid)
    R.free_tf(tid)


def test_noalloc_rejects_brick_grids_beyond_the_array(env):
    torch, native, R = env
    # 8192 x 4096 x 8 voxels, 8^3 bricks: 524,288 bricks need more than the 8 MiB array
    vol = np.zeros((8, 4096, 8192), np.uint16)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(synth.tf_random(3), 0, 4095)
    cam = synth.ortho_z_camera((8192, 4096, 8), 16, 8)
    out = torch.empty((8, 16, 4), device="cuda")
    status = _noalloc(torch, native, R, vid, tid, cam, 8, 1, out, None)
    assert status == -1  # VRC_ERR_ARG
    msg = R.lib.vrc_last_error_message(R.ctx).decode()
    assert "scratch" in msg and "maximum" in msg
    R.free_volume(vid)
    R.free_tf(tid)


def test_noalloc_kernel_choice(env):
    """kernel 0 renders with the per-ray kernel (the split render's queue would need memory,
    kernel 6 is rejected)."""
    torch, native, R = env
    vol = synth.ct_volume((40, 48, 56), seed=14)
    vid = R.upload_volume(vol)
    R.build_bricks(vid, 8)
    tid = R.set_tf(synth.tf_ct(), synth.CT_LO, synth.CT_HI)
    cam = synth.orbit_cameras(24, 1, synth.dims_of(vol), 64, 48)[0]
    ref = R.render(vid, tid, cam, ert=0.999, brick=8, kernel=1)
    out = torch.full_like(ref, float("nan"))
    native.check(R.ctx, _noalloc(torch, native, R, vid, tid, cam, 8, 0, out, None))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert _noalloc(torch, native, R, vid, tid, cam, 8, 6, out, None) == -1  # VRC_ERR_ARG
    assert "split" in R.lib.vrc_last_error_message(R.ctx).decode()
    R.free_tf(tid)
    R.free_volume(vid)
