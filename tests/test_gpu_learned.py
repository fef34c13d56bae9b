"""Learned parts end to end on the GPU.

* The unrolled, relaxed inpainting iteration through the CUDA path gives the
  same loss gradient w.r.t. the thresholds as the FP64 oracle's unrolled
  iteration (torch autograd over oracle transforms).
* The coefficient network (Sec. 4.4 residual CNN) matches the oracle forward.
* Training the threshold network briefly makes the 5-iteration hard-threshold
  loop beat the plain 5-iteration geometric schedule it was initialised to.
"""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import nn as ON

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_unrolled_iteration_gradient_matches_oracle():
    from paper_2006_04591_gb300 import learned
    from paper_2006_04591_gb300.shearlet import Bank
    from paper_2006_04591_gb300 import synth
    N, T, tau = 32, 2, 0.2
    ref = Bk.shearlet_bank(N, N, 2)
    bank = Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    K = ref["spectra"].shape[0]
    clean = synth.cartoon_texture(N, N, 5)[None]
    mask = synth.bernoulli_mask(N, N, 0.5, 6)[None]
    fm = clean * mask
    d0 = np.tile(np.array([3.0, 0.5])[None, :, None], (1, 1, K))
    d = torch.tensor(d0, dtype=torch.float32, device="cuda", requires_grad=True)
    rms = torch.tensor(ref["rms"], dtype=torch.float32, device="cuda")
    f = learned.unrolled_iht(bank, torch.tensor(fm, dtype=torch.float32, device="cuda"),
                             torch.tensor(mask, dtype=torch.uint8, device="cuda"), d, tau, rms)
    loss = ((f.double() - torch.tensor(clean, device="cuda")) ** 2).mean()
    loss.backward()
    do = torch.tensor(d0, dtype=torch.float64, requires_grad=True)
    fo = ON.unrolled_iht(torch.tensor(fm), torch.tensor(mask), torch.tensor(ref["spectra"]),
                         torch.tensor(ref["rms"]), do, tau)
    lo = ((fo - torch.tensor(clean)) ** 2).mean()
    lo.backward()
    assert abs(loss.item() - lo.item()) <= 1e-5 * lo.item()
    g, go = d.grad.double().cpu(), do.grad
    assert ((g - go).abs().max() / go.abs().max()).item() <= 1e-3


def test_coeff_net_matches_oracle():
    from paper_2006_04591_gb300 import nn
    net = nn.CoeffNet(K=17, ch=8, seed=3)
    params = {k: v.detach().double().cpu() for k, v in net.named_parameters()}
    params = {k: (v.reshape(()) if k.startswith("a") else v) for k, v in params.items()}
    c = torch.randn((2, 17, 16, 32), generator=torch.Generator().manual_seed(4))
    y = net(c.cuda())
    yo = ON.coeff_net(c.double(), params)
    assert ((y.double().cpu() - yo).abs().max() / yo.abs().max()).item() <= 1e-5


def test_short_training_beats_initial_schedule():
    from paper_2006_04591_gb300 import apps, learned, synth
    from paper_2006_04591_gb300.shearlet import Bank
    N, T = 128, 5
    bank = Bank.create(N, N, 3, device=0)
    net, hist = learned.train_thresholds(bank, steps=80, batch=4, T=T, n_pairs=200, lr=5e-3)
    init = learned.make_net(bank, T=T)
    clean, mask, masked = synth.inpaint_batch(4, N, 0.5, seed0=2000)
    ct = torch.from_numpy(clean.astype(np.float32)).cuda()
    fm = torch.from_numpy(masked.astype(np.float32)).cuda()
    mk = torch.from_numpy(mask.astype(np.float32)).cuda()
    mu8 = mk.to(torch.uint8)
    p = {}
    for name, m in [("trained", net), ("initial", init)]:
        f = learned.hard_iht(bank, fm, mu8, learned.learned_thresholds(bank, m, fm, mk))
        p[name] = apps.psnr(f, ct).mean().item()
    assert p["trained"] > p["initial"] + 0.3, p
