"""Python face of libvrc: a context object holding resident volumes, brick tables and
transfer functions, with torch tensors for device memory and torch streams for ordering.

Only marshalling happens here; every step of the method runs in the library's CUDA kernels.
Volumes are arrays of shape (nz, ny, nx) (x fastest) of uint16, int16 or float32.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import native

_DT = {np.dtype(np.uint16): native.VRC_U16, np.dtype(np.int16): native.VRC_I16,
       np.dtype(np.float32): native.VRC_F32}


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


class Renderer:
    """One libvrc context on one CUDA device."""

    def __init__(self, device: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libvrc needs a CUDA device")
        self.lib = native.load()
        self.device = int(device)
        torch.cuda.set_device(self.device)
        ctx = C.c_void_p()
        native.check(None, self.lib.vrc_create(C.byref(ctx), self.device))
        self.ctx = ctx
        self._vols = {}

    # -- lifetime -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.vrc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ck(self, status):
        native.check(self.ctx, status)

    # -- volumes --------------------------------------------------------------------------
    def upload_volume(self, vol, stream=None) -> int:
        """Makes `vol` ((nz, ny, nx) numpy array or CUDA tensor) resident; returns its id."""
        torch = _torch()
        vid = C.c_int()
        if isinstance(vol, torch.Tensor) and vol.is_cuda:
            t = vol.contiguous()
            dt = {torch.uint16: native.VRC_U16, torch.int16: native.VRC_I16,
                  torch.float32: native.VRC_F32}[t.dtype]
            nz, ny, nx = t.shape
            self._ck(self.lib.vrc_volume_upload(self.ctx, C.c_void_p(t.data_ptr()), 1, dt, nx, ny,
                                                nz, C.byref(vid), _stream_ptr(stream)))
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        else:
            a = np.ascontiguousarray(vol)
            nz, ny, nx = a.shape
            self._ck(self.lib.vrc_volume_upload(self.ctx, a.ctypes.data_as(C.c_void_p), 0,
                                                _DT[a.dtype], nx, ny, nz, C.byref(vid),
                                                _stream_ptr(stream)))
        self._vols[vid.value] = None
        return vid.value

    def update_volume(self, vol_id: int, vol, stream=None):
        """Overwrites a resident volume's values (same dtype and shape)."""
        torch = _torch()
        if isinstance(vol, torch.Tensor) and vol.is_cuda:
            t = vol.contiguous()
            self._ck(self.lib.vrc_volume_update(self.ctx, int(vol_id), C.c_void_p(t.data_ptr()), 1,
                                                _stream_ptr(stream)))
        else:
            a = np.ascontiguousarray(vol)
            self._ck(self.lib.vrc_volume_update(self.ctx, int(vol_id),
                                                a.ctypes.data_as(C.c_void_p), 0,
                                                _stream_ptr(stream)))

    def free_volume(self, vol_id: int):
        self._ck(self.lib.vrc_volume_free(self.ctx, int(vol_id)))
        self._vols.pop(vol_id, None)

    def volume_info(self, vol_id: int):
        dt, nx, ny, nz = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._ck(self.lib.vrc_volume_info(self.ctx, int(vol_id), C.byref(dt), C.byref(nx),
                                          C.byref(ny), C.byref(nz)))
        return dt.value, (nx.value, ny.value, nz.value)

    def build_bricks(self, vol_id: int, B: int, stream=None):
        self._ck(self.lib.vrc_bricks_build(self.ctx, int(vol_id), int(B), _stream_ptr(stream)))

    def bricks(self, vol_id: int, B: int, stream=None):
        """Host copies of the (min, max) brick tables, shape (nbz, nby, nbx)."""
        dt, (nx, ny, nz) = self.volume_info(vol_id)
        npdt = {native.VRC_U16: np.uint16, native.VRC_I16: np.int16, native.VRC_F32: np.float32}[dt]
        nb = tuple((n + B - 1) // B for n in (nz, ny, nx))
        mn = np.empty(nb, npdt)
        mx = np.empty(nb, npdt)
        self._ck(self.lib.vrc_bricks_get(self.ctx, int(vol_id), int(B),
                                         mn.ctypes.data_as(C.c_void_p),
                                         mx.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return mn, mx

    # -- transfer functions -----------------------------------------------------------------
    def set_tf(self, rgba, lo: float, hi: float) -> int:
        t = np.ascontiguousarray(rgba, np.float32).reshape(256, 4)
        tid = C.c_int()
        self._ck(self.lib.vrc_tf_set(self.ctx, t.ctypes.data_as(C.c_void_p), float(lo),
                                     float(hi), C.byref(tid)))
        return tid.value

    def update_tf(self, tf_id: int, rgba, lo: float, hi: float):
        t = np.ascontiguousarray(rgba, np.float32).reshape(256, 4)
        self._ck(self.lib.vrc_tf_update(self.ctx, int(tf_id), t.ctypes.data_as(C.c_void_p),
                                        float(lo), float(hi)))

    def free_tf(self, tf_id: int):
        self._ck(self.lib.vrc_tf_free(self.ctx, int(tf_id)))

    def build_occupancy(self, vol_id: int, tf_id: int, B: int, stream=None):
        self._ck(self.lib.vrc_occupancy_build(self.ctx, int(vol_id), int(tf_id), int(B),
                                              _stream_ptr(stream)))

    def occupancy(self, vol_id: int, tf_id: int, B: int, stream=None):
        _, (nx, ny, nz) = self.volume_info(vol_id)
        nb = tuple((n + B - 1) // B for n in (nz, ny, nx))
        occ = np.empty(nb, np.uint8)
        self._ck(self.lib.vrc_occupancy_get(self.ctx, int(vol_id), int(tf_id), int(B),
                                            occ.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return occ

    def cellmask(self, vol_id: int, tf_id: int, B: int, stream=None):
        """Cell transparency mask unpacked to bytes, shape (nz+1, ny+1, nx+1): entry
        [c2+1, c1+1, c0+1] is 0 when samples with floor (c0, c1, c2) have zero opacity."""
        _, (nx, ny, nz) = self.volume_info(vol_id)
        cwx = (nx + 1 + 31) // 32
        words = np.empty((nz + 1, ny + 1, cwx), np.uint32)
        self._ck(self.lib.vrc_cellmask_get(self.ctx, int(vol_id), int(tf_id), int(B),
                                           words.ctypes.data_as(C.c_void_p), words.size,
                                           _stream_ptr(stream)))
        bits = np.unpackbits(words.view(np.uint8).reshape(nz + 1, ny + 1, cwx * 4),
                             axis=-1, bitorder="little")
        return bits[..., :nx + 1].copy()

    # -- rendering ----------------------------------------------------------------------------
    def render(self, vol_id: int, tf_id: int, cam, step: float = 0.5, ert: float = 1.0,
               brick: int = 0, out=None, counters=None, stream=None, kernel: int = 0,
               interp: int = 0, preclass: int = 0, phong=None, preint: int = 0,
               ckpt=None, seg_len: int = 64):
        """Renders into a (H, W, 4) float32 CUDA tensor (allocated when `out` is None).
        `counters`: optional int64 CUDA tensor of 3 elements incremented by (nominal,
        executed, resampled) samples. `ckpt`: optional uint8 CUDA tensor of
        ckpt_bytes(...) bytes that receives the reverse-mode checkpoints (segments of
        `seg_len` samples)."""
        torch = _torch()
        if out is None:
            out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == cam.height * cam.width * 4
        cptr = None
        if counters is not None:
            assert counters.is_cuda and counters.dtype == torch.int64 and counters.numel() == 3
            cptr = C.c_void_p(counters.data_ptr())
        kptr = None
        if ckpt is not None:
            assert ckpt.is_cuda and ckpt.is_contiguous()
            kptr = C.c_void_p(ckpt.data_ptr())
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, seg_len, kernel, interp, preclass, phong,
                                  preint)
        self._ck(self.lib.vrc_render(self.ctx, int(vol_id), int(tf_id), C.byref(cs), C.byref(ps),
                                     C.c_void_p(out.data_ptr()), cptr, kptr, _stream_ptr(stream)))
        return out

    def ckpt_bytes(self, vol_id: int, cam, step: float = 0.5, seg_len: int = 64) -> int:
        """vrc_ckpt_bytes: size of the checkpoint buffer of a render of `cam`."""
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, 1.0, 0, seg_len, 0)
        n = self.lib.vrc_ckpt_bytes(C.byref(cs), C.byref(ps), int(vol_id), self.ctx)
        if n == 0:
            raise native.VrcError(-1, self.lib.vrc_last_error_message(self.ctx).decode())
        return int(n)

    def ckpt_buffer(self, vol_id: int, cam, step: float = 0.5, seg_len: int = 64):
        """A CUDA byte tensor for the checkpoints of a render of `cam` (256-byte aligned, as
        the caching allocator returns every block)."""
        torch = _torch()
        t = torch.empty(self.ckpt_bytes(vol_id, cam, step, seg_len), dtype=torch.uint8,
                        device=f"cuda:{self.device}")
        assert t.data_ptr() % 256 == 0
        return t

    def microbench(self, kind: int, stream=None) -> float:
        """vrc_microbench: 0 = FP32 flop/s, 1 = L1-hit 16-byte load bytes/s, 2 = shared-memory
        16-byte load bytes/s, measured on this context's device."""
        r = C.c_double()
        self._ck(self.lib.vrc_microbench(self.ctx, int(kind), C.byref(r), _stream_ptr(stream)))
        return r.value

    def render_host(self, vol_id: int, tf_id: int, cam, step: float = 0.5, ert: float = 1.0,
                    brick: int = 0, out=None, stream=None, kernel: int = 0,
                    interp: int = 0, preclass: int = 0, phong=None, preint: int = 0):
        """End-to-end render into host memory (pinned torch tensor or numpy array)."""
        torch = _torch()
        if out is None:
            out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32, pin_memory=True)
        ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, 64, kernel, interp, preclass, phong, preint)
        self._ck(self.lib.vrc_render_host(self.ctx, int(vol_id), int(tf_id), C.byref(cs),
                                          C.byref(ps), C.c_void_p(ptr), _stream_ptr(stream)))
        return out

    def render_host_batch(self, vol_id: int, tid: int, cams, out=None, step: float = 0.5,
                          ert: float = 1.0, brick: int = 0, stream=None, kernel: int = 0,
                          interp: int = 0, preclass: int = 0, phong=None, preint: int = 0):
        """End-to-end renders of several cameras into host memory, the read-back of each frame
        overlapping the render of the next. `out`: a list of host tensors/arrays (one per
        camera, (H, W, 4) float32) or one (n, H, W, 4) pinned tensor for equal-size cameras;
        allocated (pinned) when None."""
        torch = _torch()
        n = len(cams)
        if out is None:
            out = [torch.empty((c.height, c.width, 4), dtype=torch.float32, pin_memory=True)
                   for c in cams]
        items = [out[i] for i in range(n)]
        ptrs = (C.c_void_p * max(n, 1))(*[(t.data_ptr() if isinstance(t, torch.Tensor)
                                           else t.ctypes.data) for t in items])
        cs = (native.vrc_camera * max(n, 1))(*[native.camera_struct(c) for c in cams])
        ps = native.params_struct(step, ert, brick, 64, kernel, interp, preclass, phong, preint)
        self._ck(self.lib.vrc_render_host_batch(self.ctx, int(vol_id), int(tid), cs, n,
                                                C.byref(ps), ptrs, _stream_ptr(stream)))
        return out

    def render_backward(self, vol_id: int, tf_id: int, cam, grad_out, grad_tf, grad_vol=None,
                        step: float = 0.5, ert: float = 1.0, brick: int = 0, seg_len: int = 64,
                        stream=None, ckpt=None, kernel: int = 0, open_alpha: bool = False):
        """Adds dL/dTF to grad_tf (256x4 CUDA float32) and dL/dvoxel to grad_vol ((nz, ny, nx)
        CUDA float32, optional) for dL/dimage = grad_out ((H, W, 4) CUDA float32). `ckpt`: the
        checkpoints of a render with the same arguments (else the call renders its own).
        open_alpha: derivative from above at table opacity 0 (brick must be 0)."""
        g = grad_out.contiguous()
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, seg_len, kernel, open_alpha=open_alpha)
        self._ck(self.lib.vrc_render_backward(
            self.ctx, int(vol_id), int(tf_id), C.byref(cs), C.byref(ps), C.c_void_p(g.data_ptr()),
            C.c_void_p(ckpt.data_ptr()) if ckpt is not None else None,
            C.c_void_p(grad_tf.data_ptr()),
            C.c_void_p(grad_vol.data_ptr()) if grad_vol is not None else None,
            _stream_ptr(stream)))

    # -- object-order pieces and sort-last compositing ----------------------------------------
    def aabbs(self, vol_id: int, tf_id: int, B: int, stream=None) -> np.ndarray:
        """Tight visible box of every brick, int16 (nbz, nby, nbx, 6): (lo_x, lo_y, lo_z,
        hi_x, hi_y, hi_z) in cell coordinates, zeros when nothing in the brick is visible."""
        _, (nx, ny, nz) = self.volume_info(vol_id)
        nb = [(n + B - 1) // B for n in (nz, ny, nx)]
        out = np.empty(nb + [6], np.int16)
        self._ck(self.lib.vrc_aabbs_get(self.ctx, int(vol_id), int(tf_id), int(B),
                                        out.ctypes.data_as(C.c_void_p), nb[0] * nb[1] * nb[2],
                                        _stream_ptr(stream)))
        return out

    def build_pieces(self, vol_id: int, tf_id: int, B: int, grid, stream=None) -> int:
        """Plan of grid = (gx, gy, gz) pieces of whole bricks; returns its id."""
        g = (C.c_int * 3)(*[int(x) for x in grid])
        pid = C.c_int()
        self._ck(self.lib.vrc_pieces_build(self.ctx, int(vol_id), int(tf_id), int(B), g,
                                           C.byref(pid), _stream_ptr(stream)))
        return pid.value

    def pieces(self, plan_id: int):
        """(pieces, cuts): one dict per piece (brick_lo/hi, cell_lo/hi, vis_lo/hi, each a
        3-tuple) and the interior cut planes (x then y then z)."""
        n = C.c_int()
        self._ck(self.lib.vrc_pieces_get(self.ctx, int(plan_id), C.byref(n), None, None))
        arr = (native.vrc_piece * n.value)()
        ncut = 64 * 3
        cuts = (C.c_float * ncut)(*([float("nan")] * ncut))
        self._ck(self.lib.vrc_pieces_get(self.ctx, int(plan_id), None, arr, cuts))
        out = [{f: tuple(getattr(p, f)) for f, _ in native.vrc_piece._fields_} for p in arr]
        return out, [c for c in cuts if c == c]

    def free_pieces(self, plan_id: int):
        self._ck(self.lib.vrc_pieces_free(self.ctx, int(plan_id)))

    def render_piece(self, plan_id: int, piece: int, cam, rect, step: float = 0.5,
                     ert: float = 1.0, brick: int = 8, out=None, stream=None, kernel: int = 0,
                     interp: int = 0, preclass: int = 0, phong=None):
        """Partial image of one piece for the pixels rect = (x0, y0, w, h): a (h, w, 4)
        float32 CUDA tensor (allocated when `out` is None)."""
        torch = _torch()
        x0, y0, w, h = [int(v) for v in rect]
        if out is None:
            out = torch.empty((h, w, 4), dtype=torch.float32, device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == h * w * 4
        r = (C.c_int * 4)(x0, y0, w, h)
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, 64, kernel, interp, preclass, phong, 0)
        self._ck(self.lib.vrc_render_piece(self.ctx, int(plan_id), int(piece), C.byref(cs),
                                           C.byref(ps), r, C.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)))
        return out

    def composite(self, partials, rects, order, width: int, height: int, out=None,
                  stream=None):
        """Blends partial images (CUDA tensors, (h_k, w_k, 4) for rects[k] = (x0, y0, w, h))
        front to back in `order` into a (height, width, 4) float32 CUDA tensor."""
        torch = _torch()
        K = len(partials)
        if out is None:
            out = torch.empty((height, width, 4), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        ptrs = (C.c_void_p * max(K, 1))(*[p.data_ptr() if p is not None else None
                                          for p in partials])
        rc = (C.c_int * max(4 * K, 1))(*[int(v) for r in rects for v in r])
        od = (C.c_int * max(K, 1))(*[int(k) for k in order])
        self._ck(self.lib.vrc_composite(self.ctx, K, ptrs, rc, od, int(width), int(height),
                                        C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def render_sortlast(self, plan_id: int, cam, step: float = 0.5, ert: float = 1.0,
                        brick: int = 8, out=None, stream=None, kernel: int = 0, interp: int = 0,
                        preclass: int = 0, phong=None):
        """The image of `cam` rendered piece by piece and blended in visibility order."""
        torch = _torch()
        if out is None:
            out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == cam.height * cam.width * 4
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, 64, kernel, interp, preclass, phong, 0)
        self._ck(self.lib.vrc_render_sortlast(self.ctx, int(plan_id), C.byref(cs), C.byref(ps),
                                              C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def render_ordered(self, plan_id: int, cam, step: float = 0.5, ert: float = 1.0,
                       brick: int = 8, out=None, stream=None, kernel: int = 0, interp: int = 0,
                       preclass: int = 0, phong=None):
        """The image of `cam` rendered piece by piece front to back through one running
        image, rays terminating across pieces."""
        torch = _torch()
        if out is None:
            out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == cam.height * cam.width * 4
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, 64, kernel, interp, preclass, phong, 0)
        self._ck(self.lib.vrc_render_ordered(self.ctx, int(plan_id), C.byref(cs), C.byref(ps),
                                             C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def last_device_error(self, stream=None) -> int:
        code = C.c_int()
        self._ck(self.lib.vrc_last_device_error(self.ctx, C.byref(code), _stream_ptr(stream)))
        return code.value
