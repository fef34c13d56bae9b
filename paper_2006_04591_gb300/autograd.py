"""Differentiable shearlet layers (torch.autograd.Function over libshearlet).

ShearletDec: forward = shl_decompose (Sec. 3.4 decomposition),
             backward = shl_adjoint (its adjoint: the reconstruction without 1/W).
ShearletRec: forward = shl_reconstruct (Sec. 3.4 reconstruction),
             backward = shl_decompose with SHL_DUAL_WEIGHTED (its adjoint:
             decomposition with G_i / W).
shearlet_dec_dual: forward = shl_decompose with SHL_DUAL_WEIGHTED (the
             adjoint of the reconstruction), backward = shl_reconstruct.

Both transforms are linear, so the backward passes are exact adjoints; no
activations are saved.  Coefficients may be stored as bfloat16; gradients of
coefficients then flow in bfloat16 as well.
"""

from __future__ import annotations

import torch

from .shearlet import Bank


class _DecFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, bank: Bank, dtype):
        ctx.bank = bank
        ctx.x_dtype = x.dtype
        return bank.decompose(x.contiguous().float(), dtype=dtype)

    @staticmethod
    def backward(ctx, gc):
        gx = ctx.bank.adjoint(gc.contiguous())
        return gx.to(ctx.x_dtype), None, None


class _RecFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, bank: Bank):
        ctx.bank = bank
        ctx.c_dtype = c.dtype
        return bank.reconstruct(c.contiguous())

    @staticmethod
    def backward(ctx, gx):
        gc = ctx.bank.decompose(gx.contiguous().float(), dtype=ctx.c_dtype, dual=True)
        return gc, None


class _DualDecFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, bank: Bank):
        ctx.bank = bank
        return bank.decompose(x.contiguous().float(), dual=True)

    @staticmethod
    def backward(ctx, gc):
        return ctx.bank.reconstruct(gc.contiguous()), None


def shearlet_dec_dual(x: torch.Tensor, bank: Bank) -> torch.Tensor:
    """[B, N, M] -> [B, K, N, M]: the adjoint of shearlet_rec (float32)."""
    return _DualDecFn.apply(x, bank)


def shearlet_dec(x: torch.Tensor, bank: Bank, dtype=torch.float32) -> torch.Tensor:
    """[B, N, M] float32 -> [B, K, N, M] coefficients (float32 or bfloat16)."""
    return _DecFn.apply(x, bank, dtype)


def shearlet_rec(c: torch.Tensor, bank: Bank) -> torch.Tensor:
    """[B, K, N, M] coefficients -> [B, N, M] float32 image."""
    return _RecFn.apply(c, bank)


class ShearletDec(torch.nn.Module):
    def __init__(self, bank: Bank, dtype=torch.float32):
        super().__init__()
        self.bank = bank
        self.dtype = dtype

    def forward(self, x):
        return shearlet_dec(x, self.bank, self.dtype)


class ShearletRec(torch.nn.Module):
    def __init__(self, bank: Bank):
        super().__init__()
        self.bank = bank

    def forward(self, c):
        return shearlet_rec(c, self.bank)
