"""Differentiable rendering through torch.autograd: the forward calls vrc_render (the split
render, recording the reverse-mode checkpoints into a buffer the autograd graph keeps), the
backward vrc_render_backward (the hand-written adjoint kernel) with those checkpoints; gradients
flow to the 256 x 4 transfer function and to a float32 volume. Only argument marshalling
happens here.

    dr = DifferentiableRenderer(Renderer(0), shape=(nz, ny, nx), lo=-1024, hi=3071)
    img = dr(volume, tf, cam, step=0.5, brick=8)       # (H, W, 4) CUDA tensor
    loss = ((img - target) ** 2).sum(); loss.backward()  # volume.grad, tf.grad

The resident copies of the volume and the table are refreshed on every forward (and again in
the backward if another forward changed them in between), so several cameras can share one
loss.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native
from .renderer import _stream_ptr


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, volume, tf, dr, cam, step, ert, brick, seg_len):
        dr._load(volume, tf, brick)
        # the split render, recording its checkpoints: the adjoint differentiates exactly the
        # image it rendered (its transmittances and early-termination decisions)
        ck = dr.renderer.ckpt_buffer(dr.vol_id, cam, step, seg_len)
        img = dr.renderer.render(dr.vol_id, dr.tf_id, cam, step=step, ert=ert, brick=brick,
                                 ckpt=ck, seg_len=seg_len)
        ctx.save_for_backward(volume, tf)
        ctx.ck = ck
        ctx.dr, ctx.cam = dr, cam
        ctx.args = (step, ert, brick, seg_len)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        volume, tf = ctx.saved_tensors
        dr, cam = ctx.dr, ctx.cam
        step, ert, brick, seg_len = ctx.args
        dr._load(volume, tf, brick)  # no-op unless another forward replaced them
        R = dr.renderer
        dev = grad_img.device
        g = grad_img.detach().to(torch.float32).contiguous()
        grad_tf = torch.zeros((256, 4), dtype=torch.float32, device=dev)
        grad_vol = None
        if ctx.needs_input_grad[0]:
            grad_vol = torch.zeros(volume.shape, dtype=torch.float32, device=dev)
        cs = native.camera_struct(cam)
        ps = native.params_struct(step, ert, brick, seg_len, 0)
        R._ck(R.lib.vrc_render_backward(
            R.ctx, dr.vol_id, dr.tf_id, C.byref(cs), C.byref(ps), C.c_void_p(g.data_ptr()),
            C.c_void_p(ctx.ck.data_ptr()), C.c_void_p(grad_tf.data_ptr()),
            C.c_void_p(grad_vol.data_ptr()) if grad_vol is not None else None, _stream_ptr(None)))
        ctx.ck = None
        gtf = grad_tf.to(tf.device) if ctx.needs_input_grad[1] else None
        return grad_vol, gtf, None, None, None, None, None, None


class DifferentiableRenderer:
    """One resident float32 volume and one transfer function on a Renderer, kept in sync with
    the tensors handed to each call."""

    def __init__(self, renderer, shape, lo: float, hi: float):
        self.renderer = renderer
        self.shape = tuple(shape)
        self.lo, self.hi = float(lo), float(hi)
        self.vol_id = renderer.upload_volume(np.zeros(self.shape, np.float32))
        self.tf_id = renderer.set_tf(np.zeros((256, 4), np.float32), self.lo, self.hi)
        self._vol_key = None
        self._tf_key = None
        self._bricks = set()

    @staticmethod
    def _key(t):
        return (t.data_ptr(), t._version, tuple(t.shape))

    def _load(self, volume, tf, brick):
        R = self.renderer
        vk = self._key(volume)
        if vk != self._vol_key:
            v = volume.detach().to(torch.float32).contiguous()
            if tuple(v.shape) != self.shape:
                raise ValueError(f"volume shape {tuple(v.shape)} != {self.shape}")
            R._ck(R.lib.vrc_volume_update(R.ctx, self.vol_id, C.c_void_p(v.data_ptr()), 1,
                                          _stream_ptr(None)))
            self._vol_key = vk
            self._bricks = set()
        if brick and brick not in self._bricks:
            R.build_bricks(self.vol_id, brick)
            self._bricks.add(brick)
        tk = self._key(tf)
        if tk != self._tf_key:
            R.update_tf(self.tf_id, tf.detach().to(torch.float32).cpu().numpy(), self.lo, self.hi)
            self._tf_key = tk

    def __call__(self, volume, tf, cam, step: float = 0.5, ert: float = 1.0, brick: int = 0,
                 seg_len: int = 64):
        if not (volume.is_cuda and volume.dtype == torch.float32):
            raise TypeError("volume must be a float32 CUDA tensor of shape (nz, ny, nx)")
        return _RenderFn.apply(volume, tf, self, cam, step, ert, brick, seg_len)
