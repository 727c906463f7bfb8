"""ctypes binding of libvrc (include/vrc.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and raises ``VrcError`` on a
non-zero status. Device buffers are passed as raw pointers (``tensor.data_ptr()``) and streams
as ``torch.cuda.Stream.cuda_stream`` integers; no step of the rendering runs in Python.
The library must have been built (``paper_2005_01442_gb300.build.build()``); loading fails
loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

VRC_U16, VRC_I16, VRC_F32 = 0, 1, 2

STATUS = {0: "VRC_OK", -1: "VRC_ERR_ARG", -2: "VRC_ERR_OOM", -3: "VRC_ERR_CUDA",
          -4: "VRC_ERR_TIMEOUT", -5: "VRC_ERR_BUSY", -6: "VRC_ERR_STATE", -7: "VRC_ERR_DEVICE"}

# Every symbol include/vrc.h declares (checked by the CPU test suite).
EXPORTS = [
    "vrc_create", "vrc_destroy", "vrc_volume_upload", "vrc_volume_update", "vrc_volume_free",
    "vrc_volume_info",
    "vrc_bricks_build", "vrc_bricks_get", "vrc_tf_set", "vrc_tf_update", "vrc_tf_free",
    "vrc_occupancy_build", "vrc_occupancy_get", "vrc_cellmask_get", "vrc_render", "vrc_render_host",
    "vrc_render_noalloc", "vrc_render_backward", "vrc_server_create", "vrc_server_submit",
    "vrc_server_pump", "vrc_server_poll", "vrc_server_destroy", "vrc_last_device_error",
    "vrc_last_error_message", "vrc_status_str", "vrc_version", "vrc_aabbs_get",
    "vrc_pieces_build", "vrc_pieces_get", "vrc_pieces_free", "vrc_grid_order", "vrc_box_rect",
    "vrc_render_piece", "vrc_composite", "vrc_render_sortlast", "vrc_render_ordered",
    "vrc_render_host_batch", "vrc_ckpt_bytes", "vrc_microbench", "vrc_server_create_ex",
]


class VrcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class vrc_camera(C.Structure):
    _fields_ = [("ortho", C.c_int), ("eye", C.c_float * 3), ("center", C.c_float * 3),
                ("up", C.c_float * 3), ("fovy_deg", C.c_float), ("ortho_extent", C.c_float * 2),
                ("width", C.c_int), ("height", C.c_int)]


class vrc_params(C.Structure):
    _fields_ = [("step", C.c_float), ("ert_threshold", C.c_float), ("brick", C.c_int),
                ("seg_len", C.c_int), ("kernel", C.c_int), ("interp", C.c_int),
                ("preclass", C.c_int), ("shade", C.c_int), ("ka", C.c_float),
                ("kd", C.c_float), ("ks", C.c_float), ("shininess", C.c_float),
                ("preint", C.c_int), ("grad_open_alpha", C.c_int)]


class vrc_piece(C.Structure):
    _fields_ = [("brick_lo", C.c_int * 3), ("brick_hi", C.c_int * 3), ("cell_lo", C.c_int * 3),
                ("cell_hi", C.c_int * 3), ("vis_lo", C.c_int * 3), ("vis_hi", C.c_int * 3)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libvrc.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libvrc.so not built at {path}; run "
                               "paper_2005_01442_gb300.build.build() (needs nvcc)")
    L = C.CDLL(path)
    vp, ip, fp = C.c_void_p, C.c_int, C.c_float
    pint = C.POINTER(C.c_int)
    L.vrc_create.argtypes = [C.POINTER(vp), ip]
    L.vrc_destroy.argtypes = [vp]
    L.vrc_volume_upload.argtypes = [vp, vp, ip, ip, ip, ip, ip, pint, vp]
    L.vrc_volume_update.argtypes = [vp, ip, vp, ip, vp]
    L.vrc_volume_free.argtypes = [vp, ip]
    L.vrc_volume_info.argtypes = [vp, ip, pint, pint, pint, pint]
    L.vrc_bricks_build.argtypes = [vp, ip, ip, vp]
    L.vrc_bricks_get.argtypes = [vp, ip, ip, vp, vp, vp]
    L.vrc_tf_set.argtypes = [vp, vp, fp, fp, pint]
    L.vrc_tf_update.argtypes = [vp, ip, vp, fp, fp]
    L.vrc_tf_free.argtypes = [vp, ip]
    L.vrc_occupancy_build.argtypes = [vp, ip, ip, ip, vp]
    L.vrc_occupancy_get.argtypes = [vp, ip, ip, ip, vp, vp]
    L.vrc_cellmask_get.argtypes = [vp, ip, ip, ip, vp, C.c_long, vp]
    L.vrc_render.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp, vp, vp,
                             vp]
    L.vrc_ckpt_bytes.argtypes = [C.POINTER(vrc_camera), C.POINTER(vrc_params), ip, vp]
    L.vrc_microbench.argtypes = [vp, ip, C.POINTER(C.c_double), vp]
    L.vrc_render_host.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp, vp]
    L.vrc_render_noalloc.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp,
                                     vp, vp]
    L.vrc_render_backward.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params),
                                      vp, vp, vp, vp, vp]
    L.vrc_server_create.argtypes = [vp, ip, C.POINTER(vp)]
    L.vrc_server_create_ex.argtypes = [vp, ip, ip, C.POINTER(vp)]
    L.vrc_server_submit.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp,
                                    C.POINTER(C.c_longlong)]
    L.vrc_server_pump.argtypes = [vp, C.c_longlong, C.c_longlong, pint]
    L.vrc_server_poll.argtypes = [vp, C.c_longlong, pint]
    L.vrc_server_destroy.argtypes = [vp]
    L.vrc_aabbs_get.argtypes = [vp, ip, ip, ip, vp, C.c_long, vp]
    L.vrc_pieces_build.argtypes = [vp, ip, ip, ip, pint, pint, vp]
    L.vrc_pieces_get.argtypes = [vp, ip, pint, C.POINTER(vrc_piece), C.POINTER(C.c_float)]
    L.vrc_pieces_free.argtypes = [vp, ip]
    L.vrc_grid_order.argtypes = [C.POINTER(vrc_camera), pint, C.POINTER(C.c_float), pint]
    L.vrc_box_rect.argtypes = [C.POINTER(vrc_camera), C.POINTER(C.c_float),
                               C.POINTER(C.c_float), pint]
    L.vrc_render_piece.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params),
                                   pint, vp, vp]
    L.vrc_composite.argtypes = [vp, ip, C.POINTER(vp), pint, pint, ip, ip, vp, vp]
    L.vrc_render_sortlast.argtypes = [vp, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp,
                                      vp]
    L.vrc_render_host_batch.argtypes = [vp, ip, ip, C.POINTER(vrc_camera), ip,
                                        C.POINTER(vrc_params), C.POINTER(vp), vp]
    L.vrc_render_ordered.argtypes = [vp, ip, C.POINTER(vrc_camera), C.POINTER(vrc_params), vp,
                                     vp]
    L.vrc_last_device_error.argtypes = [vp, pint, vp]
    L.vrc_last_error_message.argtypes = [vp]
    L.vrc_last_error_message.restype = C.c_char_p
    L.vrc_status_str.argtypes = [ip]
    L.vrc_status_str.restype = C.c_char_p
    L.vrc_version.restype = ip
    for name in EXPORTS:
        if name not in ("vrc_last_error_message", "vrc_status_str", "vrc_ckpt_bytes"):
            getattr(L, name).restype = ip
    L.vrc_ckpt_bytes.restype = C.c_size_t
    _lib = L
    return L


def check(ctx, status: int):
    if status != 0:
        msg = load().vrc_last_error_message(ctx).decode() if ctx else ""
        raise VrcError(status, msg)


def camera_struct(cam) -> vrc_camera:
    c = vrc_camera()
    c.ortho = int(cam.ortho)
    c.eye[:] = [float(x) for x in cam.eye]
    c.center[:] = [float(x) for x in cam.center]
    c.up[:] = [float(x) for x in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.ortho_extent[:] = [float(x) for x in cam.ortho_extent]
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def params_struct(step=0.5, ert=1.0, brick=0, seg_len=64, kernel=0, interp=0,
                  preclass=0, phong=None, preint=0, open_alpha=False) -> vrc_params:
    """phong: None, or (ka, kd, ks, shininess) for headlight Blinn-Phong shading."""
    ka, kd, ks, shin = phong if phong is not None else (0.0, 0.0, 0.0, 1.0)
    return vrc_params(float(step), float(ert), int(brick), int(seg_len), int(kernel),
                      int(interp), int(preclass), int(phong is not None), float(ka), float(kd),
                      float(ks), float(shin), int(preint), int(bool(open_alpha)))


def grid_order(cam, grid, cuts) -> list:
    """vrc_grid_order (host only): visibility order of the pieces of a grid with interior cut
    planes `cuts` (x then y then z) for every ray of `cam`."""
    L = load()
    K = int(grid[0]) * int(grid[1]) * int(grid[2])
    g = (C.c_int * 3)(*[int(x) for x in grid])
    cu = (C.c_float * max(len(cuts), 1))(*[float(x) for x in cuts])
    order = (C.c_int * K)()
    cs = camera_struct(cam)
    st = L.vrc_grid_order(C.byref(cs), g, cu, order)
    if st != 0:
        raise VrcError(st, "vrc_grid_order")
    return list(order)


def box_rect(cam, lo, hi) -> tuple:
    """vrc_box_rect (host only): (x0, y0, w, h) of the pixels whose rays may meet [lo, hi]."""
    L = load()
    a = (C.c_float * 3)(*[float(x) for x in lo])
    b = (C.c_float * 3)(*[float(x) for x in hi])
    r = (C.c_int * 4)()
    cs = camera_struct(cam)
    st = L.vrc_box_rect(C.byref(cs), a, b, r)
    if st != 0:
        raise VrcError(st, "vrc_box_rect")
    return tuple(r)
