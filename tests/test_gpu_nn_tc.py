"""Tensor-core (tcgen05) 3x3 convolutions: the kernel rounds inputs and
weights to bfloat16 (nearest even) and accumulates in float32, so it must
equal the float64 oracle convolution of the bfloat16-rounded tensors up to
float32 summation error; the input gradient likewise with the rounded
output gradient and weights."""

import numpy as np
import pytest

from oracle import nn as ON

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5


def _rel(a, b):
    a = a.detach().double().cpu()
    b = b.detach().double().cpu()
    return ((a - b).abs().max() / b.abs().max().clamp_min(1e-30)).item()


def _bf(t):
    return t.to(torch.bfloat16).double()


# the last six take the wide tiles: up to 112 input channels with at most 32
# outputs, or at most 32 inputs with up to 112 outputs (padded channels zero)
SHAPES = [(2, 33, 32, 5, 128), (1, 32, 33, 4, 256), (2, 2, 32, 3, 128), (1, 16, 16, 3, 384),
          (1, 48, 48, 2, 128), (3, 32, 32, 1, 128), (1, 7, 5, 6, 256),
          (1, 102, 32, 3, 128), (2, 32, 85, 2, 128), (1, 85, 32, 2, 128), (1, 32, 102, 2, 128),
          (1, 64, 16, 2, 128), (1, 16, 60, 2, 256),
          # widths that are not multiples of 128 (ragged last tile) or of 4
          # (float2 loads): the dual networks' 30 x 182 sinograms and others
          (2, 7, 32, 30, 182), (1, 32, 5, 4, 182), (1, 16, 16, 3, 200), (1, 8, 32, 2, 130),
          (1, 32, 32, 5, 64), (1, 4, 16, 3, 18)]


@pytest.mark.parametrize("B,Ci,Co,H,W", SHAPES)
def test_tc_forward_matches_rounded_oracle(B, Ci, Co, H, W):
    from paper_2006_04591_gb300 import nn
    assert nn.shl_nn_conv3x3_tc_supported(Ci, Co, H, W)
    gen = torch.Generator().manual_seed(B * 1000 + Ci * 10 + Co)
    x = torch.randn((B, Ci, H, W), generator=gen)
    w = torch.randn((Co, Ci, 3, 3), generator=gen) * 0.2
    b = torch.randn(Co, generator=gen)
    out = torch.empty((B, Co, H, W), device="cuda")
    nn.shl_nn_conv3x3_forward_tc(x.cuda(), w.cuda(), b.cuda(), out)
    nn.shl_nn_tc_status()
    want = ON.conv3x3(_bf(x), _bf(w), b.double())
    assert _rel(out, want) <= TOL


@pytest.mark.parametrize("B,Ci,Co,H,W", SHAPES)
def test_tc_backward_data_matches_rounded_oracle(B, Ci, Co, H, W):
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(B * 7 + Ci + Co * 3)
    w = torch.randn((Co, Ci, 3, 3), generator=gen) * 0.2
    gout = torch.randn((B, Co, H, W), generator=gen)
    gin = torch.empty((B, Ci, H, W), device="cuda")
    nn.shl_nn_conv3x3_backward_data_tc(gout.cuda(), w.cuda(), gin)
    nn.shl_nn_tc_status()
    xo = torch.zeros((B, Ci, H, W), dtype=torch.float64, requires_grad=True)
    yo = ON.conv3x3(xo, _bf(w), torch.zeros(Co, dtype=torch.float64))
    (yo * _bf(gout)).sum().backward()
    assert _rel(gin, xo.grad) <= TOL


WSHAPES = [(2, 33, 32, 5, 128), (1, 32, 33, 4, 256), (2, 2, 32, 3, 128), (1, 42, 48, 2, 128),
           (3, 32, 16, 1, 128), (1, 7, 5, 6, 256), (1, 32, 85, 3, 128), (2, 16, 96, 2, 128),
           (1, 42, 60, 2, 256), (2, 7, 32, 30, 182), (1, 32, 5, 4, 182), (1, 16, 16, 3, 200),
           (1, 32, 32, 2, 64), (1, 4, 8, 3, 18)]


@pytest.mark.parametrize("B,Ci,Co,H,W", WSHAPES)
def test_tc_weight_gradient_matches_rounded_oracle(B, Ci, Co, H, W):
    from paper_2006_04591_gb300 import nn
    assert nn.shl_nn_conv3x3_wgrad_tc_supported(Ci, Co, H, W)
    gen = torch.Generator().manual_seed(B * 31 + Ci * 7 + Co)
    x = torch.randn((B, Ci, H, W), generator=gen)
    gout = torch.randn((B, Co, H, W), generator=gen)
    gw = torch.empty((Co, Ci, 3, 3), device="cuda")
    gb = torch.empty(Co, device="cuda")
    nn.shl_nn_conv3x3_backward_weight_tc(x.cuda(), gout.cuda(), gw, gb)
    nn.shl_nn_tc_status()
    want = torch.nn.grad.conv2d_weight(_bf(x), (Co, Ci, 3, 3), _bf(gout), padding=1)
    assert _rel(gw, want) <= 1e-4
    assert _rel(gb, gout.double().sum((0, 2, 3))) <= 1e-5


def test_tc_rejects_unsupported_shapes():
    from paper_2006_04591_gb300 import nn
    from paper_2006_04591_gb300.shearlet import ShearletError
    assert not nn.shl_nn_conv3x3_tc_supported(32, 32, 8, 181)      # odd width
    assert not nn.shl_nn_conv3x3_tc_supported(32, 32, 8, 14)       # narrower than 16
    assert not nn.shl_nn_conv3x3_tc_supported(120, 32, 8, 128)     # more than 112 inputs
    assert not nn.shl_nn_conv3x3_tc_supported(64, 64, 8, 128)      # wide on both sides
    assert not nn.shl_nn_conv3x3_tc_supported(48, 80, 8, 128)
    assert not nn.shl_nn_conv3x3_tc_supported(32, 120, 8, 128)
    assert not nn.shl_nn_conv3x3_wgrad_tc_supported(43, 32, 8, 128)
    assert not nn.shl_nn_conv3x3_wgrad_tc_supported(32, 97, 8, 128)
    assert not nn.shl_nn_conv3x3_wgrad_tc_supported(32, 32, 8, 99)
    x = torch.zeros((1, 32, 8, 101), device="cuda")
    with pytest.raises(ShearletError):
        nn.shl_nn_conv3x3_forward_tc(x, torch.zeros((32, 32, 3, 3), device="cuda"), None,
                                     torch.empty_like(x))


class _RoundedConv(torch.autograd.Function):
    """float64 reference of what the tensor-core path computes: the forward
    and both gradients see bfloat16-rounded operands (the bias gradient the
    unrounded output gradient)."""

    @staticmethod
    def forward(ctx, x, w, b):
        ctx.save_for_backward(x, w)
        return ON.conv3x3(_bf(x), _bf(w), b)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        F = torch.nn.grad
        gin = F.conv2d_input(x.shape, _bf(w), _bf(g), padding=1)
        gw = F.conv2d_weight(_bf(x), w.shape, _bf(g), padding=1)
        return gin, gw, g.sum((0, 2, 3))


def test_coeff_net_tc_matches_rounded_reference():
    """The residual coefficient network with tensor-core convolutions against
    a float64 network that rounds the same operands to bfloat16: output and
    first-layer weight gradient agree to float32 level (the bfloat16 rounding
    itself moves that gradient by ~2 % relative L2 here, so a comparison with
    the float32 path could not tell a layout error from rounding)."""
    from paper_2006_04591_gb300 import nn
    c = torch.randn((2, 33, 8, 128), generator=torch.Generator().manual_seed(9))
    net = nn.CoeffNet(K=33, ch=32, seed=5, tc=True)
    y = net(c.cuda())
    (y * y).sum().backward()
    nn.shl_nn_tc_status()
    P = {k: v.detach().double().cpu() for k, v in net.named_parameters()}
    w0 = P["w0"].clone().requires_grad_(True)
    pr = lambda h, a: torch.where(h >= 0, h, a * h)
    h = pr(_RoundedConv.apply(c.double(), w0, P["b0"]), P["a0"])
    h = pr(_RoundedConv.apply(h, P["w1"], P["b1"]), P["a1"])
    yo = c.double() + _RoundedConv.apply(h, P["w2"], P["b2"])
    (yo * yo).sum().backward()
    l2 = lambda a, b: ((a.detach().double().cpu() - b).norm() / b.norm()).item()
    assert l2(y, yo) <= 1e-4
    assert l2(net.w0.grad, w0.grad) <= 1e-3


WS_CHILD = """
import torch
from oracle import nn as ON
from paper_2006_04591_gb300 import nn
def bf(t): return t.to(torch.bfloat16).double()
for (B, Ci, Co, H, W) in [(2, 33, 32, 5, 128), (1, 32, 48, 9, 256), (1, 2, 16, 3, 128)]:
    g = torch.Generator().manual_seed(B * 7 + Ci + H)
    x = torch.randn((B, Ci, H, W), generator=g)
    w = torch.randn((Co, Ci, 3, 3), generator=g) * 0.2
    b = torch.randn(Co, generator=g)
    out = torch.empty((B, Co, H, W), device="cuda")
    nn.shl_nn_conv3x3_forward_tc(x.cuda(), w.cuda(), b.cuda(), out)
    nn.shl_nn_tc_status()
    want = ON.conv3x3(bf(x), bf(w), b.double())
    err = ((out.double().cpu() - want).abs().max() / want.abs().max()).item()
    assert err <= 2e-5, (B, Ci, Co, H, W, err)
print("ws ok")
"""


def test_warp_specialised_conv_matches_rounded_oracle():
    """The opt-in warp-specialised forward kernel (SHL_CONV_WS=1), in a child
    process: producers, MMA issuer and epilogue handing rows over through
    mbarriers give the rounded oracle's result."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    env["SHL_CONV_WS"] = "1"
    r = subprocess.run([sys.executable, "-c", WS_CHILD], cwd=root, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ws ok" in r.stdout


@pytest.mark.parametrize("tc,B,Ci,Co,H,W", [
    ("grouped", 2, 102, 32, 3, 128), ("grouped", 1, 32, 85, 4, 128),
    ("grouped", 1, 102, 85, 2, 256), ("grouped", 2, 7, 32, 3, 256),
    (True, 2, 102, 32, 3, 128), (True, 1, 32, 85, 4, 128), (True, 2, 85, 32, 2, 128),
    (True, 2, 7, 32, 30, 182), ("grouped", 1, 102, 32, 3, 182)])
def test_wide_tc_conv_autograd_matches_rounded_oracle(tc, B, Ci, Co, H, W):
    # the shearlet-domain primal layers of the learned primal-dual
    # reconstruction (102 -> 32, 32 -> 85): tc=True takes them in one call per
    # pass on the wide tiles (the weight gradient of 102 inputs in groups of
    # 42), tc="grouped" in channel groups of at most 48
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(Ci * 100 + Co)
    x = torch.randn((B, Ci, H, W), generator=gen)
    w = torch.randn((Co, Ci, 3, 3), generator=gen) * 0.1
    b = torch.randn(Co, generator=gen)
    go = torch.randn((B, Co, H, W), generator=gen)
    xg = x.cuda().requires_grad_(True)
    wg = w.cuda().requires_grad_(True)
    bg = b.cuda().requires_grad_(True)
    y = nn.conv3x3(xg, wg, bg, tc=tc)
    (y * go.cuda()).sum().backward()
    nn.shl_nn_tc_status()
    assert _rel(y, ON.conv3x3(_bf(x), _bf(w), b.double())) <= TOL
    # input gradient: rounded gout and w; weight gradient: rounded x and gout
    xo = torch.zeros((B, Ci, H, W), dtype=torch.float64, requires_grad=True)
    (ON.conv3x3(xo, _bf(w), torch.zeros(Co, dtype=torch.float64)) * _bf(go)).sum().backward()
    assert _rel(xg.grad, xo.grad) <= TOL
    wo = torch.zeros((Co, Ci, 3, 3), dtype=torch.float64, requires_grad=True)
    (ON.conv3x3(_bf(x), wo, None) * _bf(go)).sum().backward()
    assert _rel(wg.grad, wo.grad) <= TOL
    # the bias gradient sums the float32 (unrounded) output gradient
    assert _rel(bg.grad, go.double().sum((0, 2, 3))) <= 1e-5
