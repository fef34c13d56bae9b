"""Learned parts on the GPU: binding of include/shearlet_nn.h, autograd
Functions whose forward and backward run in libshearlet's kernels, the two
networks and Adam.

* ThresholdNet - predicts per-subband thresholds delta_{t,i} (t < T, i < K)
  of the unrolled inpainting iteration (Sec. 4.3) from [f_masked, mask]:
  avgpool -> 4 x (3x3 conv + PReLU) -> global average pool -> linear ->
  softplus.
* CoeffNet - residual 3-layer CNN on shearlet coefficients after the learned
  proximal operators of Sec. 4.4: c + W3 A W2 A W1 c, PReLU A.

Both networks run their 3x3 convolutions (forward, input and weight
gradients) on the tensor cores (tcgen05, bfloat16 operands, float32 accumulation) wherever the
shape allows it (tc=True, the default), else on the float32 kernels.

torch only provides tensors (memory), parameter containers and the autograd
tape; every arithmetic step calls the library.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import shearlet as S

_sig_done = False


def lib():
    global _sig_done
    L = S.lib()
    if not _sig_done:
        vp, i, f, ll, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong, ctypes.c_size_t
        sig = {
            "shl_nn_last_error": (ctypes.c_char_p, []),
            "shl_nn_conv3x3_forward": (i, [vp, vp, vp, vp, i, i, i, i, i, vp]),
            "shl_nn_conv3x3_workspace_floats": (sz, [i, i, i, i, i]),
            "shl_nn_conv3x3_backward_data": (i, [vp, vp, vp, i, i, i, i, i, vp, vp]),
            "shl_nn_conv3x3_backward_weight": (i, [vp, vp, vp, vp, i, i, i, i, i, vp, vp]),
            "shl_nn_conv3x3_tc_supported": (i, [i, i, i, i]),
            "shl_nn_conv3x3_forward_tc": (i, [vp, vp, vp, vp, i, i, i, i, i, vp]),
            "shl_nn_conv3x3_backward_data_tc": (i, [vp, vp, vp, i, i, i, i, i, vp]),
            "shl_nn_tc_status": (i, [vp]),
            "shl_nn_conv3x3_wgrad_tc_supported": (i, [i, i, i, i]),
            "shl_nn_conv3x3_backward_weight_tc_workspace_floats": (sz, [i, i, i, i, i]),
            "shl_nn_conv3x3_backward_weight_tc": (i, [vp, vp, vp, vp, i, i, i, i, i, vp, vp]),
            "shl_nn_tc_last_error": (ctypes.c_char_p, []),
            "shl_nn_prelu_forward": (i, [vp, vp, vp, ll, vp]),
            "shl_nn_reduce_workspace_floats": (sz, [ll]),
            "shl_nn_prelu_backward": (i, [vp, vp, vp, vp, vp, ll, vp, vp]),
            "shl_nn_avgpool": (i, [vp, vp, i, i, i, i, i, vp]),
            "shl_nn_gap_forward": (i, [vp, vp, i, i, i, vp]),
            "shl_nn_gap_backward": (i, [vp, vp, i, i, i, vp]),
            "shl_nn_linear_forward": (i, [vp, vp, vp, vp, i, i, i, vp]),
            "shl_nn_linear_backward": (i, [vp, vp, vp, vp, vp, vp, i, i, i, vp]),
            "shl_nn_softplus_forward": (i, [vp, vp, ll, vp]),
            "shl_nn_softplus_backward": (i, [vp, vp, vp, ll, vp]),
            "shl_nn_gate_forward": (i, [vp, i, vp, vp, i, f, vp, i, ll, vp]),
            "shl_nn_gate_workspace_floats": (sz, [i]),
            "shl_nn_gate_backward": (i, [vp, vp, vp, i, f, vp, vp, vp, i, ll, vp, vp]),
            "shl_nn_mse_forward": (i, [vp, vp, vp, ll, vp, vp]),
            "shl_nn_mse_backward": (i, [vp, vp, vp, vp, ll, vp]),
            "shl_nn_adam": (i, [vp, vp, vp, vp, ll, f, f, f, f, i, vp]),
            "shl_nn_mask_mix": (i, [vp, vp, vp, vp, ll, vp]),
            "shl_nn_mask_mix_backward": (i, [vp, vp, vp, ll, vp]),
            "shl_nn_cast": (i, [vp, i, vp, ll, vp]),
            "shl_nn_axpy": (i, [vp, f, vp, ll, vp]),
            "shl_nn_scale_thresholds": (i, [vp, vp, vp, i, i, i, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sig_done = True
    return L


def _chk(name, st):
    if st != 0:
        raise S.ShearletError(name, st, lib().shl_nn_last_error().decode())


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _st(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ws(n, like):
    return torch.empty(max(int(n), 1), dtype=torch.float32, device=like.device)


# ----------------------------------------------------------- C-named calls
def shl_nn_conv3x3_forward(x, w, b, out):
    B, Ci, H, W = x.shape
    _chk("conv3x3_forward", lib().shl_nn_conv3x3_forward(_p(x), _p(w), _p(b), _p(out), B, Ci,
                                                          w.shape[0], H, W, _st(x)))


def _chk_tc(name, st):
    if st != 0:
        raise S.ShearletError(name, st, lib().shl_nn_tc_last_error().decode())


def shl_nn_conv3x3_tc_supported(Ci, Co, H, W):
    return bool(lib().shl_nn_conv3x3_tc_supported(Ci, Co, H, W))


def shl_nn_conv3x3_forward_tc(x, w, b, out):
    B, Ci, H, W = x.shape
    _chk_tc("conv3x3_forward_tc", lib().shl_nn_conv3x3_forward_tc(
        _p(x), _p(w), _p(b), _p(out), B, Ci, w.shape[0], H, W, _st(x)))


def shl_nn_conv3x3_backward_data_tc(gout, w, gin):
    B, Ci, H, W = gin.shape
    _chk_tc("conv3x3_backward_data_tc", lib().shl_nn_conv3x3_backward_data_tc(
        _p(gout), _p(w), _p(gin), B, Ci, w.shape[0], H, W, _st(gin)))


def shl_nn_conv3x3_wgrad_tc_supported(Ci, Co, H, W):
    return bool(lib().shl_nn_conv3x3_wgrad_tc_supported(Ci, Co, H, W))


def shl_nn_conv3x3_backward_weight_tc(x, gout, gw, gb):
    B, Ci, H, W = x.shape
    Co = gout.shape[1]
    L = lib()
    ws = _ws(L.shl_nn_conv3x3_backward_weight_tc_workspace_floats(B, Ci, Co, H, W), x)
    _chk_tc("conv3x3_backward_weight_tc", L.shl_nn_conv3x3_backward_weight_tc(
        _p(x), _p(gout), _p(gw), _p(gb), B, Ci, Co, H, W, _p(ws), _st(x)))


def shl_nn_tc_status(stream=None):
    s = ctypes.c_void_p(None if stream is None else stream.cuda_stream)
    _chk_tc("tc_status", lib().shl_nn_tc_status(s))


def shl_nn_conv3x3_backward(x, w, gout, need_gin=True, tc=False, tc_w=False):
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    L = lib()
    gw = torch.empty_like(w)
    gb = torch.empty(Co, dtype=torch.float32, device=x.device)
    if tc_w and Ci <= TC_WCH:
        shl_nn_conv3x3_backward_weight_tc(x, gout, gw, gb)
    elif tc_w:
        # one call stages at most 42 input channels (3 Ci <= 128 rows); the
        # weight gradient of an input-channel group depends on that group only
        for k, (c0, c1) in enumerate(_groups(Ci, TC_WCH)):
            gwg = torch.empty((Co, c1 - c0, 3, 3), dtype=torch.float32, device=x.device)
            gbg = torch.empty(Co, dtype=torch.float32, device=x.device)
            shl_nn_conv3x3_backward_weight_tc(x[:, c0:c1].contiguous(), gout, gwg, gbg)
            gw[:, c0:c1] = gwg
            if k == 0:
                gb.copy_(gbg)
    ws = _ws(L.shl_nn_conv3x3_workspace_floats(B, Ci, Co, H, W), x) if (not tc_w or
                                                                      (need_gin and not tc)) else None
    if not tc_w and Ci <= 64:
        _chk("conv3x3_backward_weight", L.shl_nn_conv3x3_backward_weight(
            _p(x), _p(gout), _p(gw), _p(gb), B, Ci, Co, H, W, _p(ws), _st(x)))
    elif not tc_w:
        # the kernel stages at most 64 input channels of a tile; the weight
        # gradient of an input-channel group depends on that group only
        for c0 in range(0, Ci, 64):
            c1 = min(Ci, c0 + 64)
            xg = x[:, c0:c1].contiguous()
            gwg = torch.empty((Co, c1 - c0, 3, 3), dtype=torch.float32, device=x.device)
            wsg = _ws(L.shl_nn_conv3x3_workspace_floats(B, c1 - c0, Co, H, W), x)
            _chk("conv3x3_backward_weight", L.shl_nn_conv3x3_backward_weight(
                _p(xg), _p(gout), _p(gwg), _p(gb), B, c1 - c0, Co, H, W, _p(wsg), _st(x)))
            gw[:, c0:c1] = gwg
    gin = None
    if need_gin:
        gin = torch.empty_like(x)
        if tc:
            shl_nn_conv3x3_backward_data_tc(gout, w, gin)
        else:
            _chk("conv3x3_backward_data", L.shl_nn_conv3x3_backward_data(
                _p(gout), _p(w), _p(gin), B, Ci, Co, H, W, _p(ws), _st(x)))
    return gin, gw, gb


# ------------------------------------------------------------- autograd
# Channel groups for the tensor-core kernels (conv3x3(..., tc="grouped")):
# one call takes at most 48 input and 48 output channels (weight gradient: 42
# input channels, 3 Ci <= 128).  Wider layers run as a sum over input-channel
# groups (partials added by shl_nn_axpy) for each output-channel group; a
# layer within the limits is a single call.
TC_CH, TC_WCH = 48, 42


def _groups(n, g):
    return [(a, min(n, a + g)) for a in range(0, n, g)]


def _tc_width_ok(H, W):
    return H >= 1 and W >= 16 and W % 2 == 0


def _axpy(src, dst, alpha=1.0):
    _chk("axpy", lib().shl_nn_axpy(_p(src), float(alpha), _p(dst), src.numel(), _st(dst)))


def conv3x3_forward_tc_grouped(x, w, b, out):
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    cig, cog = _groups(Ci, TC_CH), _groups(Co, TC_CH)
    xs = [x if len(cig) == 1 else x[:, a:c].contiguous() for a, c in cig]
    for o0, o1 in cog:
        dst = out if len(cog) == 1 else torch.empty((B, o1 - o0, H, W), device=x.device)
        for k, (a, c) in enumerate(cig):
            wg = w[o0:o1, a:c].contiguous()
            if k == 0:
                shl_nn_conv3x3_forward_tc(xs[k], wg, b[o0:o1].contiguous(), dst)
            else:
                part = torch.empty_like(dst)
                shl_nn_conv3x3_forward_tc(xs[k], wg, None, part)
                _axpy(part, dst)
        if len(cog) > 1:
            out[:, o0:o1] = dst


def conv3x3_backward_data_tc_grouped(gout, w, gin):
    B, Ci, H, W = gin.shape
    Co = w.shape[0]
    cig, cog = _groups(Ci, TC_CH), _groups(Co, TC_CH)
    gos = [gout if len(cog) == 1 else gout[:, o0:o1].contiguous() for o0, o1 in cog]
    for a, c in cig:
        dst = gin if len(cig) == 1 else torch.empty((B, c - a, H, W), device=gin.device)
        for k, (o0, o1) in enumerate(cog):
            wg = w[o0:o1, a:c].contiguous()
            if k == 0:
                shl_nn_conv3x3_backward_data_tc(gos[k], wg, dst)
            else:
                part = torch.empty_like(dst)
                shl_nn_conv3x3_backward_data_tc(gos[k], wg, part)
                _axpy(part, dst)
        if len(cig) > 1:
            gin[:, a:c] = dst


def conv3x3_backward_weight_tc_grouped(x, gout, gw, gb):
    Ci, Co = x.shape[1], gout.shape[1]
    cig, cog = _groups(Ci, TC_WCH), _groups(Co, TC_CH)
    if len(cig) == 1 and len(cog) == 1:
        shl_nn_conv3x3_backward_weight_tc(x, gout, gw, gb)
        return
    xs = [x[:, a:c].contiguous() for a, c in cig]
    for o0, o1 in cog:
        go = gout[:, o0:o1].contiguous()
        for k, (a, c) in enumerate(cig):
            gwg = torch.empty((o1 - o0, c - a, 3, 3), device=x.device)
            gbg = torch.empty(o1 - o0, device=x.device)
            shl_nn_conv3x3_backward_weight_tc(xs[k], go, gwg, gbg)
            gw[o0:o1, a:c] = gwg
            if k == 0:
                gb[o0:o1] = gbg


class _Conv3x3(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, tc):
        x = x.contiguous()
        out = torch.empty((x.shape[0], w.shape[0], x.shape[2], x.shape[3]), dtype=torch.float32,
                          device=x.device)
        B, Ci, H, W = x.shape
        Co = w.shape[0]
        ctx.grouped = tc == "grouped" and _tc_width_ok(H, W)
        if ctx.grouped:
            # every pass on the tensor cores, in channel groups
            conv3x3_forward_tc_grouped(x, w.contiguous(), b.contiguous(), out)
            ctx.save_for_backward(x, w)
            return out
        # tensor cores for each pass where one call takes the shape
        ctx.tc_fwd = bool(tc) and shl_nn_conv3x3_tc_supported(Ci, Co, H, W)
        ctx.tc_bwd = bool(tc) and shl_nn_conv3x3_tc_supported(Co, Ci, H, W)
        ctx.tc_w = bool(tc) and shl_nn_conv3x3_wgrad_tc_supported(min(Ci, TC_WCH), Co, H, W)
        if ctx.tc_fwd:
            shl_nn_conv3x3_forward_tc(x, w.contiguous(), b.contiguous(), out)
        else:
            shl_nn_conv3x3_forward(x, w.contiguous(), b.contiguous(), out)
        ctx.save_for_backward(x, w)
        return out

    @staticmethod
    def backward(ctx, gout):
        x, w = ctx.saved_tensors
        gout = gout.contiguous()
        w = w.contiguous()
        if not ctx.grouped:
            gin, gw, gb = shl_nn_conv3x3_backward(x, w, gout, ctx.needs_input_grad[0],
                                                 tc=ctx.tc_bwd, tc_w=ctx.tc_w)
            return gin, gw, gb, None
        gw = torch.empty_like(w)
        gb = torch.empty(w.shape[0], dtype=torch.float32, device=x.device)
        conv3x3_backward_weight_tc_grouped(x, gout, gw, gb)
        gin = None
        if ctx.needs_input_grad[0]:
            gin = torch.empty_like(x)
            conv3x3_backward_data_tc_grouped(gout, w, gin)
        return gin, gw, gb, None


class _PReLU(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, a):
        x = x.contiguous()
        y = torch.empty_like(x)
        _chk("prelu_forward", lib().shl_nn_prelu_forward(_p(x), _p(a), _p(y), x.numel(), _st(x)))
        ctx.save_for_backward(x, a)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, a = ctx.saved_tensors
        gx = torch.empty_like(x)
        ga = torch.empty(1, dtype=torch.float32, device=x.device)
        ws = _ws(lib().shl_nn_reduce_workspace_floats(x.numel()), x)
        _chk("prelu_backward", lib().shl_nn_prelu_backward(_p(x), _p(a), _p(gy.contiguous()), _p(gx),
                                                            _p(ga), x.numel(), _p(ws), _st(x)))
        return gx, ga.reshape(a.shape)


class _GAP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        B, C, H, W = x.shape
        y = torch.empty((B, C), dtype=torch.float32, device=x.device)
        _chk("gap_forward", lib().shl_nn_gap_forward(_p(x.contiguous()), _p(y), B, C, H * W, _st(x)))
        ctx.shape = x.shape
        return y

    @staticmethod
    def backward(ctx, gy):
        B, C, H, W = ctx.shape
        gx = torch.empty(ctx.shape, dtype=torch.float32, device=gy.device)
        _chk("gap_backward", lib().shl_nn_gap_backward(_p(gy.contiguous()), _p(gx), B, C, H * W, _st(gy)))
        return gx


class _Linear(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b):
        B, I = x.shape
        O = w.shape[0]
        y = torch.empty((B, O), dtype=torch.float32, device=x.device)
        _chk("linear_forward", lib().shl_nn_linear_forward(_p(x.contiguous()), _p(w), _p(b), _p(y), B, I, O, _st(x)))
        ctx.save_for_backward(x, w)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, w = ctx.saved_tensors
        B, I = x.shape
        O = w.shape[0]
        gx = torch.empty_like(x)
        gw = torch.empty_like(w)
        gb = torch.empty(O, dtype=torch.float32, device=x.device)
        _chk("linear_backward", lib().shl_nn_linear_backward(_p(x.contiguous()), _p(w), _p(gy.contiguous()), _p(gx),
                                                              _p(gw), _p(gb), B, I, O, _st(x)))
        return gx, gw, gb


class _Softplus(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        x = x.contiguous()
        y = torch.empty_like(x)
        _chk("softplus_forward", lib().shl_nn_softplus_forward(_p(x), _p(y), x.numel(), _st(x)))
        ctx.save_for_backward(x)
        return y

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        gx = torch.empty_like(x)
        _chk("softplus_backward", lib().shl_nn_softplus_backward(_p(x), _p(gy.contiguous()), _p(gx), x.numel(), _st(x)))
        return gx


class _Gate(torch.autograd.Function):
    """Relaxed hard threshold on [B, K, H, W] float32 coefficients with
    thresholds delta [B, K] (times scale [K] if given)."""

    @staticmethod
    def forward(ctx, c, delta, scale, tau):
        assert c.dtype == torch.float32, "gate takes float32 coefficients"
        c = c.contiguous()
        delta = delta.contiguous()
        B, K, H, W = c.shape
        y = torch.empty(c.shape, dtype=torch.float32, device=c.device)
        _chk("gate_forward", lib().shl_nn_gate_forward(_p(c), 0, _p(delta), _p(scale), K,
                                                        float(tau), _p(y), B * K, H * W, _st(c)))
        ctx.save_for_backward(c, delta)
        ctx.scale = scale
        ctx.tau = float(tau)
        return y

    @staticmethod
    def backward(ctx, gy):
        c, delta = ctx.saved_tensors
        B, K, H, W = c.shape
        gc = torch.empty_like(c)
        gd = torch.empty_like(delta)
        ws = _ws(lib().shl_nn_gate_workspace_floats(B * K), c)
        _chk("gate_backward", lib().shl_nn_gate_backward(_p(c), _p(delta), _p(ctx.scale), K, ctx.tau,
                                                          _p(gy.contiguous()), _p(gc), _p(gd), B * K,
                                                          H * W, _p(ws), _st(c)))
        return gc, gd, None, None


class _MaskMix(torch.autograd.Function):
    """u = mask (f_masked - f) + f, differentiable in f."""

    @staticmethod
    def forward(ctx, f_masked, mask_u8, f):
        u = torch.empty_like(f)
        _chk("mask_mix", lib().shl_nn_mask_mix(_p(f_masked.contiguous()), _p(mask_u8), _p(f.contiguous()), _p(u),
                                                f.numel(), _st(f)))
        ctx.save_for_backward(mask_u8)
        return u

    @staticmethod
    def backward(ctx, gu):
        (mask_u8,) = ctx.saved_tensors
        gf = torch.empty_like(gu)
        _chk("mask_mix_backward", lib().shl_nn_mask_mix_backward(_p(mask_u8), _p(gu.contiguous()), _p(gf),
                                                                  gu.numel(), _st(gu)))
        return None, None, gf


class _MSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b):
        a, b = a.contiguous(), b.contiguous()
        out = torch.empty(1, dtype=torch.float32, device=a.device)
        ws = _ws(lib().shl_nn_reduce_workspace_floats(a.numel()), a)
        _chk("mse_forward", lib().shl_nn_mse_forward(_p(a), _p(b), _p(out), a.numel(), _p(ws), _st(a)))
        ctx.save_for_backward(a, b)
        return (out / a.numel()).reshape(())

    @staticmethod
    def backward(ctx, g):
        a, b = ctx.saved_tensors
        ga = torch.empty_like(a)
        gs = g.reshape(1).contiguous().float()
        _chk("mse_backward", lib().shl_nn_mse_backward(_p(a), _p(b), _p(gs), _p(ga), a.numel(), _st(a)))
        return ga, None


class _ResidualAdd(torch.autograd.Function):
    """c + h with h overwritten in place (h is a fresh convolution output that
    nothing saved), the sum done by shl_nn_axpy."""

    @staticmethod
    def forward(ctx, c, h):
        c = c.contiguous()
        _chk("axpy", lib().shl_nn_axpy(_p(c), 1.0, _p(h), h.numel(), _st(h)))
        ctx.mark_dirty(h)
        return h

    @staticmethod
    def backward(ctx, g):
        return g, g


class _Scale(torch.autograd.Function):
    """alpha * x (a python float alpha) through shl_nn_axpy into zeros."""

    @staticmethod
    def forward(ctx, x, alpha):
        ctx.alpha = float(alpha)
        x = x.contiguous()
        y = torch.zeros_like(x)
        _chk("axpy", lib().shl_nn_axpy(_p(x), ctx.alpha, _p(y), x.numel(), _st(x)))
        return y

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gx = torch.zeros_like(g)
        _chk("axpy", lib().shl_nn_axpy(_p(g), ctx.alpha, _p(gx), g.numel(), _st(g)))
        return gx, None


def conv3x3(x, w, b, tc=False):
    """3x3 convolution; tc=True runs the forward, the input gradient and the
    weight gradient on the tensor cores (bfloat16 operands, float32
    accumulation) where one call takes the shape, else the float32 kernels;
    tc="grouped" runs every pass on the tensor cores whenever the row width
    is even (at least 16), in channel groups for wider layers (measured slower
    for the learned primal-dual networks, whose steps are bound by launches)."""
    return _Conv3x3.apply(x, w, b, tc)


def prelu(x, a):
    return _PReLU.apply(x, a)


def gap(x):
    return _GAP.apply(x)


def linear(x, w, b):
    return _Linear.apply(x, w, b)


def softplus(x):
    return _Softplus.apply(x)


def gate(c, delta, tau, scale=None):
    return _Gate.apply(c, delta, scale, tau)


def mask_mix(f_masked, mask_u8, f):
    return _MaskMix.apply(f_masked, mask_u8, f)


def mse(a, b):
    return _MSE.apply(a, b)


def scale_thresholds(d, scale, out):
    """out[t][b][k] = d[b][t][k] * scale[k] (no grad)."""
    B, T, K = d.shape
    _chk("scale_thresholds", lib().shl_nn_scale_thresholds(_p(d.contiguous()), _p(scale), _p(out), B, T, K, _st(d)))
    return out


def avgpool(x, f):
    B, C, H, W = x.shape
    y = torch.empty((B, C, H // f, W // f), dtype=torch.float32, device=x.device)
    _chk("avgpool", lib().shl_nn_avgpool(_p(x.contiguous()), _p(y), B, C, H, W, f, _st(x)))
    return y


def to_float(c):
    """bfloat16 -> float32 through the library's cast kernel (no grad)."""
    y = torch.empty(c.shape, dtype=torch.float32, device=c.device)
    _chk("cast", lib().shl_nn_cast(_p(c.contiguous()), 1, _p(y), c.numel(), _st(c)))
    return y


class _ToFloat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c):
        return to_float(c)

    @staticmethod
    def backward(ctx, g):
        y = torch.empty(g.shape, dtype=torch.bfloat16, device=g.device)
        _chk("cast", lib().shl_nn_cast(_p(g.contiguous()), 0, _p(y), g.numel(), _st(g)))
        return y


def bf16_to_float(c):
    return _ToFloat.apply(c)


# ---------------------------------------------------------------- models
def _init_conv(co, ci, gen, device):
    std = math.sqrt(2.0 / (ci * 9))
    w = torch.randn((co, ci, 3, 3), generator=gen) * std
    return w.to(device).requires_grad_(True), torch.zeros(co, device=device, requires_grad=True)


class ThresholdNet(torch.nn.Module):
    """[B, 2, H, W] (f_masked, mask) -> thresholds [B, T, K] (relative to RMS_i)."""

    def __init__(self, K, T=10, ch=32, pool=4, seed=0, device="cuda", scale=1.0, tc=True):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        self.K, self.T, self.pool, self.tc = K, T, pool, tc
        chans = [2, ch, ch, ch, ch]
        for l in range(4):
            w, b = _init_conv(chans[l + 1], chans[l], g, device)
            setattr(self, "w%d" % l, torch.nn.Parameter(w.detach()))
            setattr(self, "b%d" % l, torch.nn.Parameter(b.detach()))
            setattr(self, "a%d" % l, torch.nn.Parameter(torch.full((1,), 0.25, device=device)))
        self.wl = torch.nn.Parameter((torch.randn((T * K, ch), generator=g) * 0.01).to(device))
        self.bl = torch.nn.Parameter(torch.full((T * K,), float(scale), device=device))

    def forward(self, x):
        h = avgpool(x, self.pool) if self.pool > 1 else x
        for l in range(4):
            h = prelu(conv3x3(h, getattr(self, "w%d" % l), getattr(self, "b%d" % l), self.tc),
                      getattr(self, "a%d" % l))
        y = softplus(linear(gap(h), self.wl, self.bl))
        return y.reshape(x.shape[0], self.T, self.K)


class CoeffNet(torch.nn.Module):
    """c + W3 A W2 A W1 c on [B, K, H, W] float32 coefficients."""

    def __init__(self, K, ch=32, seed=0, device="cuda", tc=True):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        self.tc = tc
        chans = [K, ch, ch, K]
        for l in range(3):
            w, b = _init_conv(chans[l + 1], chans[l], g, device)
            if l == 2:
                w = w * 0.1
            setattr(self, "w%d" % l, torch.nn.Parameter(w.detach()))
            setattr(self, "b%d" % l, torch.nn.Parameter(b.detach()))
        self.a0 = torch.nn.Parameter(torch.full((1,), 0.25, device=device))
        self.a1 = torch.nn.Parameter(torch.full((1,), 0.25, device=device))

    def forward(self, c):
        h = prelu(conv3x3(c, self.w0, self.b0, self.tc), self.a0)
        h = prelu(conv3x3(h, self.w1, self.b1, self.tc), self.a1)
        return _ResidualAdd.apply(c, conv3x3(h, self.w2, self.b2, self.tc))


@torch.no_grad()
def clip_grad_norm(params, max_norm):
    """Scale the gradients of ``params`` so that their global 2-norm is at
    most ``max_norm``; returns the norm before clipping.  The gradients are
    gathered into one flat buffer; its sum of squares comes from
    shl_nn_mse_forward against zeros and the scaling from shl_nn_axpy (the
    parameters' gradients then become views of the scaled buffer)."""
    L = lib()
    ps = [p for p in params if p.grad is not None]
    if not ps:
        return 0.0
    flat = torch.cat([p.grad.reshape(-1) for p in ps])
    n = flat.numel()
    zero = torch.zeros_like(flat)
    sq = torch.empty(1, dtype=torch.float32, device=flat.device)
    ws = _ws(L.shl_nn_reduce_workspace_floats(n), flat)
    _chk("mse_forward", L.shl_nn_mse_forward(_p(flat), _p(zero), _p(sq), n, _p(ws), _st(flat)))
    total = math.sqrt(float(sq.item()))
    if total > max_norm:
        _chk("axpy", L.shl_nn_axpy(_p(flat), max_norm / total, _p(zero), n, _st(flat)))
        off = 0
        for p in ps:
            k = p.grad.numel()
            p.grad = zero[off:off + k].view_as(p.grad)
            off += k
    return total


CHECKPOINT_VERSION = 1


def save_checkpoint(path, module, opt=None, step=0, meta=None):
    """Versioned checkpoint: the module's parameters and buffers, the Adam
    state (moments, step count, hyper-parameters) and free-form metadata,
    written atomically (temporary file, then rename)."""
    import os
    state = {"version": CHECKPOINT_VERSION, "step": int(step), "meta": meta or {},
             "module": {k: v.detach().cpu() for k, v in module.state_dict().items()}}
    if opt is not None:
        state["adam"] = {"m": [m.cpu() for m in opt.m], "v": [v.cpu() for v in opt.v],
                         "step_count": opt.step_count, "lr": opt.lr, "b1": opt.b1,
                         "b2": opt.b2, "eps": opt.eps}
    tmp = "%s.%d.tmp" % (path, os.getpid())
    torch.save(state, tmp)
    os.replace(tmp, path)


def load_checkpoint(path, module, opt=None):
    """Restore a checkpoint written by save_checkpoint into ``module`` (and
    ``opt``); returns (step, meta).  Raises ValueError on a version or shape
    mismatch."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    if state.get("version") != CHECKPOINT_VERSION:
        raise ValueError("checkpoint version %r, expected %d" % (state.get("version"),
                                                                CHECKPOINT_VERSION))
    own = module.state_dict()
    if set(own) != set(state["module"]) or any(own[k].shape != state["module"][k].shape
                                               for k in own):
        raise ValueError("checkpoint does not match the module's parameters")
    module.load_state_dict(state["module"])
    if opt is not None and "adam" in state:
        a = state["adam"]
        if len(a["m"]) != len(opt.m):
            raise ValueError("checkpoint optimiser state does not match")
        with torch.no_grad():
            for dst, src in zip(opt.m + opt.v, a["m"] + a["v"]):
                dst.copy_(src)
        opt.step_count, opt.lr, opt.b1, opt.b2, opt.eps = (a["step_count"], a["lr"], a["b1"],
                                                           a["b2"], a["eps"])
    return state["step"], state["meta"]


class Adam:
    """Adam over a list of parameters; the update runs in shl_nn_adam."""

    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.params = [p for p in params]
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0

    def zero_grad(self):
        for p in self.params:
            p.grad = None

    @torch.no_grad()
    def step(self):
        self.step_count += 1
        for p, m, v in zip(self.params, self.m, self.v):
            if p.grad is None:
                continue
            _chk("adam", lib().shl_nn_adam(_p(p), _p(p.grad.contiguous()), _p(m), _p(v), p.numel(),
                                            self.lr, self.b1, self.b2, self.eps, self.step_count,
                                            _st(p)))
