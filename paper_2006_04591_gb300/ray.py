"""Binding of the parallel-beam ray transform (``include/shearlet_ray.h``).

``RayTransform(n, n_angles, n_det)`` wraps ``shl_ray_create``; ``forward``
and ``adjoint`` call ``shl_ray_forward`` / ``shl_ray_adjoint`` on the
current stream.  ``ray_forward`` / ``ray_adjoint`` are the same operators as
autograd functions (each one's backward is the other), for the learned
primal-dual reconstruction of Sec. 4.4.  All arithmetic runs in the CUDA
kernels of ``csrc/ray.cu``.
"""

from __future__ import annotations

import ctypes
import math

import torch

from .shearlet import _check, _ptr, _stream, lib


class RayTransform:
    """Joseph-method parallel-beam transform of n x n images on [-1, 1]^2 at
    angles pi a / n_angles and n_det bins over [-sqrt 2, sqrt 2]."""

    def __init__(self, n: int, n_angles: int = 30, n_det: int | None = None, device: int = 0):
        self.n, self.n_angles = n, n_angles
        self.n_det = n_det if n_det is not None else int(math.ceil(math.sqrt(2.0) * n))
        self.device = device
        h = ctypes.c_void_p()
        _check("shl_ray_create", lib().shl_ray_create(n, n_angles, self.n_det, device,
                                                      ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle is not None:
            _check("shl_ray_destroy", lib().shl_ray_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, t, shape):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if tuple(t.shape[1:]) != shape:
            raise ValueError("expected shape [B, %s], got %s" % (", ".join(map(str, shape)),
                                                                  tuple(t.shape)))

    def forward(self, img, out=None):
        img = img.contiguous()
        self._chk(img, (self.n, self.n))
        B = img.shape[0]
        out = out if out is not None else torch.empty((B, self.n_angles, self.n_det),
                                                      device=img.device)
        _check("shl_ray_forward", lib().shl_ray_forward(self.handle, _ptr(img), B, _ptr(out),
                                                        _stream(None, img.device)))
        return out

    def adjoint(self, sino, out=None):
        sino = sino.contiguous()
        self._chk(sino, (self.n_angles, self.n_det))
        B = sino.shape[0]
        out = out if out is not None else torch.empty((B, self.n, self.n), device=sino.device)
        _check("shl_ray_adjoint", lib().shl_ray_adjoint(self.handle, _ptr(sino), B, _ptr(out),
                                                        _stream(None, sino.device)))
        return out

    def norm(self, iters: int = 30, seed: int = 0) -> float:
        """||R||_2 by power iteration on R^T R."""
        g = torch.Generator(device="cuda").manual_seed(seed)
        x = torch.rand((1, self.n, self.n), device="cuda", generator=g)
        lam = 0.0
        for _ in range(iters):
            y = self.adjoint(self.forward(x))
            lam = y.norm().item()
            x = y / lam
        return math.sqrt(lam)


class _Fwd(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return op.forward(x)

    @staticmethod
    def backward(ctx, g):
        return ctx.op.adjoint(g.contiguous()), None


class _Adj(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, op):
        ctx.op = op
        return op.adjoint(y)

    @staticmethod
    def backward(ctx, g):
        return ctx.op.forward(g.contiguous()), None


def ray_forward(x, op: RayTransform):
    """R x with backward R^T."""
    return _Fwd.apply(x, op)


def ray_adjoint(y, op: RayTransform):
    """R^T y with backward R."""
    return _Adj.apply(y, op)
