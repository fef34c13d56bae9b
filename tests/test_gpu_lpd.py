"""GPU parity of the learned primal-dual network (Sec. 4.4, Algorithm 2)
against the FP64 oracle (``oracle/lpd.py``), image and shearlet domain.

Weights and the operator scale are drawn or computed on the oracle side
(seeded numpy, float64 power iteration) and loaded into both networks; the
GPU network runs its float32 convolutions (tc=False) so that the comparison
is float32 against float64: outputs within 1e-4 and parameter gradients
within 1e-3 of their largest magnitude.
"""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import lpd as OL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, A, D, ITERS, NP, ND, CH = 32, 8, 46, 3, 2, 2, 8


def _setup(domain, seed=0):
    from paper_2006_04591_gb300.lpd import LPD
    from paper_2006_04591_gb300.ray import RayTransform
    from paper_2006_04591_gb300.shearlet import Bank
    ref = Bk.shearlet_bank(N, N, 1) if domain == "shearlet" else None
    op_o = OL.Operator(N, A, D, G=None if ref is None else ref["spectra"])
    scale = 1.0 / OL.op_norm(op_o)
    op_o.scale = scale
    bank = Bank.from_spectra(ref["spectra"], ref["idx"], device=0) if ref is not None else None
    net = LPD(RayTransform(N, A, D, device=0), domain, bank, iters=ITERS, n_primal=NP,
              n_dual=ND, ch=CH, tc=False, scale=scale)
    rng = np.random.default_rng(seed)
    primal, dual = [], []
    for mods, out in ((net.primal, primal), (net.dual, dual)):
        for m in mods:
            d = {}
            for name, p in m.named_parameters():
                if name.startswith("a"):
                    v = rng.uniform(0.1, 0.4, p.shape)
                elif name.startswith("b"):
                    v = rng.normal(0, 0.05, p.shape)
                else:
                    v = rng.normal(0, np.sqrt(2.0 / (p.shape[1] * 9)), p.shape)
                with torch.no_grad():
                    p.copy_(torch.from_numpy(v).float())
                d[name] = torch.tensor(v, dtype=torch.float64, requires_grad=True)
            out.append(d)
    return net, op_o, primal, dual


@pytest.mark.parametrize("domain", ["image", "shearlet"])
def test_lpd_forward_and_gradients_match_oracle(domain):
    net, op_o, primal, dual = _setup(domain)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((2, A, D))
    target = rng.random((2, N, N))
    # oracle
    out_o = OL.lpd(torch.as_tensor(g), op_o, primal, dual, NP, ND)
    torch.mean((out_o - torch.as_tensor(target)) ** 2).backward()
    # GPU
    from paper_2006_04591_gb300 import nn as NN
    gt = torch.from_numpy(g).float().cuda()
    tt = torch.from_numpy(target).float().cuda()
    out = net(gt)
    NN.mse(out, tt).backward()
    o, w = out.detach().cpu().numpy(), out_o.detach().numpy()
    assert np.abs(o - w).max() <= 1e-4 * np.abs(w).max()
    for mods, ref in ((net.primal, primal), (net.dual, dual)):
        for i in (0, ITERS - 1):
            for name in ("w0", "w2", "b1", "a0"):
                gg = getattr(mods[i], name).grad.cpu().numpy()
                gr = ref[i][name].grad.numpy()
                assert np.abs(gg - gr).max() <= 1e-3 * max(np.abs(gr).max(), 1e-12), (i, name)


def test_lpd_training_reduces_loss():
    from paper_2006_04591_gb300 import lpd as L
    net, op, bank, hist, ts = L.train("shearlet", steps=40, batch=2, N=128, n_train=16,
                                      log_every=39)
    assert hist[-1][1] < 0.5 * hist[0][1]
    ev = L.evaluate(net, op)
    assert np.isfinite(ev["psnr"]) and ev["psnr"] > 10.0


def test_weight_gradient_with_more_than_64_input_channels():
    # the shearlet-domain primal network's first layer has (Np + 1) K = 102
    # input channels: the float32 weight gradient runs in channel groups
    from oracle import nn as ON
    from paper_2006_04591_gb300 import nn as NN
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 102, 20, 24))
    w = rng.standard_normal((8, 102, 3, 3)) * 0.05
    b = rng.standard_normal(8) * 0.1
    go = rng.standard_normal((2, 8, 20, 24))
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    (ON.conv3x3(xt, wt, bt) * torch.as_tensor(go)).sum().backward()
    xg = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    wg = torch.tensor(w, dtype=torch.float32, device="cuda", requires_grad=True)
    bg = torch.tensor(b, dtype=torch.float32, device="cuda", requires_grad=True)
    (NN.conv3x3(xg, wg, bg) * torch.tensor(go, dtype=torch.float32, device="cuda")).sum().backward()
    for got, want in ((wg.grad, wt.grad), (bg.grad, bt.grad), (xg.grad, xt.grad)):
        g, r = got.cpu().numpy(), want.numpy()
        assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max()


def test_clip_grad_norm():
    from paper_2006_04591_gb300 import nn as NN
    g = torch.Generator(device="cuda").manual_seed(0)
    ps = [torch.nn.Parameter(torch.zeros(s, device="cuda")) for s in ((3, 5), (7,), (2, 2, 3, 3))]
    for p in ps:
        p.grad = torch.randn(p.shape, device="cuda", generator=g)
    want = np.sqrt(sum(float((p.grad.double() ** 2).sum()) for p in ps))
    before = [p.grad.clone() for p in ps]
    assert abs(NN.clip_grad_norm(ps, 10 * want) - want) <= 1e-5 * want
    assert all(torch.equal(a, p.grad) for a, p in zip(before, ps))     # below the limit
    NN.clip_grad_norm(ps, 0.5)
    after = np.sqrt(sum(float((p.grad.double() ** 2).sum()) for p in ps))
    assert abs(after - 0.5) <= 1e-5


@pytest.mark.parametrize("domain", ["image", "shearlet"])
def test_graph_training_step_equals_eager(domain):
    """Forward and backward replayed as one CUDA graph compute what the eager
    step computes (every kernel of the step is deterministic): after five
    steps (one eager, four replays, clipping and Adam in between) the
    parameters and the logged losses are the same bits as five eager steps."""
    from paper_2006_04591_gb300 import lpd
    runs = []
    for graph in (False, True):
        net, op, bank, hist, ts = lpd.train(domain, steps=5, n_train=8, log_every=1, graph=graph)
        runs.append(([p.detach().clone() for p in net.parameters()], hist))
    (pa, ha), (pb, hb) = runs
    assert ha == hb
    assert all(torch.equal(a, b) for a, b in zip(pa, pb))
