"""GPU kernels of the learned parts against the FP64 oracle (oracle/nn.py):
forward values and gradients (through torch's autograd tape calling our
kernels) on seeded inputs, float32 tolerance 1e-5 relative to max."""

import numpy as np
import pytest

from oracle import nn as ON

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    a = a.detach().double().cpu()
    b = b.detach().double().cpu()
    return ((a - b).abs().max() / b.abs().max().clamp_min(1e-30)).item()


def _pair(t, grad=True):
    """float32 CUDA leaf and float64 CPU leaf with the same values."""
    g = t.float().cuda().clone().requires_grad_(grad)
    o = t.double().clone().requires_grad_(grad)
    return g, o


@pytest.mark.parametrize("B,Ci,Co,H,W", [(2, 3, 5, 17, 70), (1, 33, 32, 24, 40), (2, 32, 33, 16, 64),
                                         (3, 2, 8, 9, 9)])
def test_conv3x3_forward_and_gradients(B, Ci, Co, H, W):
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(B * 100 + Ci)
    x, xo = _pair(torch.randn((B, Ci, H, W), generator=gen))
    w, wo = _pair(torch.randn((Co, Ci, 3, 3), generator=gen) * 0.2)
    b, bo = _pair(torch.randn(Co, generator=gen))
    y = nn.conv3x3(x, w, b)
    yo = ON.conv3x3(xo, wo, bo)
    assert _rel(y, yo) <= TOL
    gy = torch.randn(yo.shape, generator=gen)
    (y * gy.cuda()).sum().backward()
    (yo * gy.double()).sum().backward()
    assert _rel(x.grad, xo.grad) <= TOL
    assert _rel(w.grad, wo.grad) <= TOL
    assert _rel(b.grad, bo.grad) <= TOL


def test_prelu_gap_linear_softplus_chain():
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(7)
    x, xo = _pair(torch.randn((3, 4, 8, 8), generator=gen))
    a, ao = _pair(torch.tensor([0.2]))
    w, wo = _pair(torch.randn((6, 4), generator=gen))
    b, bo = _pair(torch.randn(6, generator=gen))
    y = nn.softplus(nn.linear(nn.gap(nn.prelu(x, a)), w, b))
    yo = ON.softplus(ON.linear(ON.gap(ON.prelu(xo, ao)), wo, bo))
    assert _rel(y, yo) <= TOL
    gy = torch.randn(yo.shape, generator=gen)
    (y * gy.cuda()).sum().backward()
    (yo * gy.double()).sum().backward()
    for g, o in [(x, xo), (a, ao), (w, wo), (b, bo)]:
        assert _rel(g.grad, o.grad) <= TOL


def test_gate_mse_and_mask_mix():
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(9)
    c, co = _pair(torch.randn((2, 3, 16, 16), generator=gen))
    d, do = _pair(torch.rand((2, 3), generator=gen) + 0.2)
    y = nn.gate(c, d, 0.1)
    yo = ON.gate(co, do, 0.1)
    assert _rel(y, yo) <= TOL
    t = torch.randn(yo.shape, generator=gen)
    l = nn.mse(y, t.float().cuda())
    lo = ON.mse(yo, t.double())
    assert abs(l.item() - lo.item()) <= TOL * lo.item()
    l.backward()
    lo.backward()
    assert _rel(c.grad, co.grad) <= TOL and _rel(d.grad, do.grad) <= TOL
    fm = torch.randn((2, 16, 16), generator=gen).cuda()
    m = (torch.rand((2, 16, 16), generator=gen) < 0.5).to(torch.uint8).cuda()
    f = torch.randn((2, 16, 16), generator=gen).cuda().requires_grad_(True)
    u = nn.mask_mix(fm, m, f)
    assert torch.equal(u, torch.where(m.bool(), fm, f))
    u.sum().backward()
    assert torch.equal(f.grad, (1 - m).float())


def test_avgpool_and_cast():
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(11)
    x = torch.randn((2, 2, 16, 12), generator=gen)
    assert _rel(nn.avgpool(x.cuda(), 4), ON.avgpool(x.double(), 4)) <= TOL
    h = x.bfloat16().cuda()
    assert torch.equal(nn.to_float(h), h.float())


def test_adam_matches_oracle_over_steps():
    from paper_2006_04591_gb300 import nn
    gen = torch.Generator().manual_seed(12)
    p0 = torch.randn(100, generator=gen)
    p = p0.clone().cuda().requires_grad_(True)
    opt = nn.Adam([p], lr=1e-2)
    po, m, v = p0.double(), torch.zeros(100, dtype=torch.float64), torch.zeros(100, dtype=torch.float64)
    for s in range(1, 6):
        g = torch.randn(100, generator=gen)
        p.grad = g.cuda()
        opt.step()
        po, m, v = ON.adam_step(po, g.double(), m, v, s, 1e-2)
    assert _rel(p, po) <= 1e-6


def test_threshold_net_matches_oracle():
    from paper_2006_04591_gb300 import nn
    net = nn.ThresholdNet(K=5, T=3, ch=8, pool=2, seed=1)
    params = {k: v.detach().double().cpu().clone().requires_grad_(True) for k, v in net.named_parameters()}
    params = {k: (v.reshape(()) if k.startswith("a") else v) for k, v in params.items()}
    gen = torch.Generator().manual_seed(13)
    x = torch.randn((2, 2, 16, 16), generator=gen)
    y = net(x.cuda())
    yo = ON.threshold_net(x.double(), params, 2).reshape(2, 3, 5)
    assert _rel(y, yo) <= TOL
