"""FP64 oracle for the learned parts: the small convolutional networks and the
relaxed (differentiable) hard threshold used to train per-subband thresholds.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Forward definitions are written out with plain float64 torch CPU tensor
operations; gradients come from torch's autograd on these definitions.

* 3x3 convolution with zero padding 1 (the affine maps W_{w,b} of the
  learned proximal operators, Sec. 4.4): out[b, o] = bias[o] +
  sum_{i, dy, dx} w[o, i, dy, dx] in[b, i, y + dy - 1, x + dx - 1].
* PReLU: x for x >= 0 and a x otherwise.  Sec. 4.4 writes the negative branch
  as -c x; a = -c.
* average pooling by an integer factor, global average pooling, a linear
  layer, softplus log(1 + e^x).
* relaxed hard threshold ("gate"): c * sigmoid((|c| / delta - 1) / tau), a
  scale-free relaxation (tau is relative to the threshold) that tends to the
  hard threshold T_delta of Sec. 4.2 as tau -> 0.
* mean squared error and one Adam step (Kingma and Ba 2015, with bias
  correction).
"""

from __future__ import annotations

import numpy as np
import torch

F64 = torch.float64


def t64(a):
    return torch.as_tensor(np.asarray(a), dtype=F64)


def conv3x3(x, w, b=None):
    """x [B, Ci, H, W], w [Co, Ci, 3, 3], b [Co] -> [B, Co, H, W]."""
    B, Ci, H, W = x.shape
    xp = torch.zeros((B, Ci, H + 2, W + 2), dtype=x.dtype)
    xp[:, :, 1:-1, 1:-1] = x
    out = torch.zeros((B, w.shape[0], H, W), dtype=x.dtype)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + W]
            out = out + torch.einsum("oi,bihw->bohw", w[:, :, dy, dx], patch)
    if b is not None:
        out = out + b[None, :, None, None]
    return out


def prelu(x, a):
    return torch.where(x >= 0, x, a * x)


def avgpool(x, f):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // f, f, W // f, f).mean(dim=(3, 5))


def gap(x):
    return x.mean(dim=(2, 3))


def linear(x, w, b):
    return x @ w.T + b


def softplus(x):
    return torch.log1p(torch.exp(-torch.abs(x))) + torch.clamp(x, min=0)


def gate(c, delta, tau):
    """c [B, K, H, W], delta [B, K]."""
    return c * torch.sigmoid((torch.abs(c) / delta[:, :, None, None] - 1.0) / tau)


def mse(a, b):
    return torch.mean((a - b) ** 2)


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Returns updated (p, m, v) after one Adam step (step counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (torch.sqrt(vh) + eps), m, v


def threshold_net(x, params, pool):
    """The threshold predictor: avgpool -> 4 x (conv3x3 + PReLU) -> global
    average pool -> linear -> softplus.  x [B, 2, H, W] -> [B, P]."""
    h = avgpool(x, pool) if pool > 1 else x
    for l in range(4):
        h = prelu(conv3x3(h, params["w%d" % l], params["b%d" % l]), params["a%d" % l])
    return softplus(linear(gap(h), params["wl"], params["bl"]))


def coeff_net(c, params):
    """Residual 3-layer CNN on coefficients: c + W3 A W2 A W1 c (Sec. 4.4)."""
    h = prelu(conv3x3(c, params["w0"], params["b0"]), params["a0"])
    h = prelu(conv3x3(h, params["w1"], params["b1"]), params["a1"])
    return c + conv3x3(h, params["w2"], params["b2"])


# ------------------------------------------- transforms with autograd (torch)
def dec_t(x, G):
    """Natural-order decomposition c_i = ifft2(fft2(x) G_i) (Sec. 3.4 with the
    shifts cancelled, as oracle.transform.decompose_natural), torch float64,
    differentiable.  x [B, N, M], G [K, N, M] real -> [B, K, N, M] real."""
    X = torch.fft.fft2(x.to(torch.complex128))
    return torch.fft.ifft2(X[:, None] * G[None]).real


def rec_t(c, G, weights=True):
    """ifft2(sum_i G_i fft2(c_i) [/ W]) (Sec. 3.4 reconstruction), differentiable."""
    acc = torch.sum(G[None] * torch.fft.fft2(c.to(torch.complex128)), dim=1)
    if weights:
        acc = acc / torch.sum(G ** 2, dim=0)[None]
    return torch.fft.ifft2(acc).real


def unrolled_iht(f_masked, mask, G, rms, deltas, tau):
    """Unrolled inpainting iteration with the relaxed threshold: for each t,
    u = mask (f_masked - f) + f, f = rec(gate(dec(u), deltas[:, t] * rms)).
    deltas [B, T, K] relative to RMS_i; returns the final f."""
    f = torch.zeros_like(f_masked)
    for t in range(deltas.shape[1]):
        u = mask * (f_masked - f) + f
        c = dec_t(u, G)
        f = rec_t(gate(c, deltas[:, t] * rms[None], tau), G)
    return f
