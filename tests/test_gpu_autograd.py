"""GPU backward passes of the shearlet layers against the FP64 oracle's
adjoints, plus directional finite differences through the GPU path."""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def setup():
    from paper_2006_04591_gb300.shearlet import Bank
    ref = Bk.shearlet_bank(64, 64, 3)
    return ref, Bank.from_spectra(ref["spectra"], ref["idx"], device=0)


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("bf16", 1e-2)])
def test_dec_backward_is_oracle_adjoint(setup, dtype, tol):
    from paper_2006_04591_gb300.autograd import shearlet_dec
    ref, bank = setup
    K = ref["spectra"].shape[0]
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal((2, 64, 64)).astype(np.float32)).cuda()
    x.requires_grad_(True)
    w = rng.standard_normal((2, K, 64, 64)).astype(np.float32)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    c = shearlet_dec(x, bank, tdt)
    assert c.dtype == tdt
    wt = torch.from_numpy(w).cuda().to(tdt)
    (c.float() * wt.float()).sum().backward()
    want = np.stack([OT.adjoint(wt[b].float().cpu().numpy().astype(np.float64), ref["psi_hat"]).real
                     for b in range(2)])
    assert _rel(x.grad.cpu().numpy(), want) <= tol


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("bf16", 1e-2)])
def test_rec_backward_is_oracle_dual_decomposition(setup, dtype, tol):
    from paper_2006_04591_gb300.autograd import shearlet_rec
    ref, bank = setup
    K = ref["spectra"].shape[0]
    rng = np.random.default_rng(2)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    c = torch.from_numpy(rng.standard_normal((2, K, 64, 64)).astype(np.float32)).cuda().to(tdt)
    c.requires_grad_(True)
    w = rng.standard_normal((2, 64, 64)).astype(np.float32)
    y = shearlet_rec(c, bank)
    (y * torch.from_numpy(w).cuda()).sum().backward()
    assert c.grad.dtype == tdt
    want = np.stack([OT.decompose_dual(w[b].astype(np.float64), ref["psi_hat"]).real
                     for b in range(2)])
    assert _rel(c.grad.float().cpu().numpy(), want) <= tol


def test_directional_finite_difference_through_gpu_path(setup):
    from paper_2006_04591_gb300.autograd import shearlet_dec, shearlet_rec
    ref, bank = setup
    K = ref["spectra"].shape[0]
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn((1, 64, 64), generator=g).cuda().requires_grad_(True)
    w = torch.randn((1, K, 64, 64), generator=g).cuda()
    # quadratic loss ||rec(dec(x) * w)||^2, reduced in float64: its central
    # difference is exact for any step, so a wide step keeps float32
    # rounding of the transforms out of the quotient
    loss = lambda z: (shearlet_rec(shearlet_dec(z, bank) * w, bank).double() ** 2).sum()
    loss(x).backward()
    eps = 1e-1
    for _ in range(3):
        v = torch.randn((1, 64, 64), generator=g).cuda()
        with torch.no_grad():
            fd = (loss(x + eps * v) - loss(x - eps * v)).double() / (2 * eps)
        an = (x.grad.double() * v.double()).sum()
        # directional derivative: compare on the Cauchy-Schwarz scale |grad| |v|
        assert abs(fd - an) <= 1e-5 * (x.grad.double().norm() * v.double().norm())
