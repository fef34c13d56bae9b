"""Parity at the shapes of the five workloads (the benchmark runs config 2's
transform; these check the others at their own sizes).  Large batches are
run in one call exactly as a user would, and checked on sampled images /
subbands that the FP64 oracle computes one by one."""

import numpy as np
import pytest

from oracle import apps as OA
from oracle import bank as Bk
from oracle import transform as OT
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 1e-2


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / np.abs(b).max()


def _bank(n, J):
    from paper_2006_04591_gb300.shearlet import Bank
    ref = Bk.shearlet_bank(n, n, J)
    return ref, Bank.from_spectra(ref["spectra"], ref["idx"], device=0)


def test_config1_plain_transform_256_k17():
    """One 256 x 256 image (8 ellipses + noise), 2 scales, 17 filters:
    decomposition, reconstruction, adjoint identity and perfect reconstruction."""
    ref, bank = _bank(256, 2)
    assert bank.K == 17
    x64 = synth.plain_transform_image(256, seed=1)
    x = x64.astype(np.float32)[None]
    xt = torch.from_numpy(x).cuda()
    c = bank.decompose(xt)
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    assert _rel(c.cpu().numpy(), want) <= TOL32
    r = bank.reconstruct(c).cpu().numpy()
    assert np.abs(r - x).max() <= TOL32 * np.abs(x).max()
    rng = np.random.default_rng(2)
    w = rng.standard_normal((1, 17, 256, 256)).astype(np.float32)
    adj = bank.adjoint(torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)
    lhs = np.sum(c.cpu().numpy().astype(np.float64) * w)
    rhs = np.sum(x.astype(np.float64) * adj)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_config2_denoise_16x512_k49():
    """16 noisy 512 x 512 cartoons in one call, 49 filters, threshold
    3 sigma RMS_i; two sampled images against the oracle's PSNR."""
    from paper_2006_04591_gb300 import apps
    sigma = 30 / 255
    ref, bank = _bank(512, 4)
    assert bank.K == 49
    clean, noisy = synth.denoise_batch(16, 512, sigma, seed0=100)
    den = apps.denoise(bank, torch.from_numpy(noisy.astype(np.float32)).cuda(), sigma, 3.0)
    den = den.cpu().numpy()
    d = OA.subband_thresholds(ref["rms"], ref["idx"], sigma, 3.0)
    for b in (0, 15):
        want = OA.denoise(noisy[b].astype(np.float32).astype(np.float64), ref["psi_hat"], d)
        assert abs(OA.psnr(clean[b], den[b]) - OA.psnr(clean[b], want)) < 0.05


def test_config3_layer_32x256_k33_bf16():
    """Batch 32 of 256 x 256, 33 filters, bfloat16 coefficients: forward and
    the adjoint backward against the oracle on sampled images."""
    from paper_2006_04591_gb300.autograd import shearlet_dec
    ref, bank = _bank(256, 3)
    assert bank.K == 33
    clean, noisy = synth.denoise_batch(32, 256, 30 / 255, seed0=1000)
    x = torch.from_numpy(noisy.astype(np.float32)).cuda().requires_grad_(True)
    c = shearlet_dec(x, bank, torch.bfloat16)
    rng = np.random.default_rng(4)
    w = torch.from_numpy(rng.standard_normal((32, 33, 256, 256)).astype(np.float32)).cuda()
    (c.float() * w).sum().backward()
    for b in (0, 31):
        want, _ = OT.decompose_batch(noisy[b:b + 1].astype(np.float32), ref["psi_hat"])
        assert _rel(c[b].detach().float().cpu().numpy(), want[0]) <= TOL16
        wb = w[b].to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
        gwant = OT.adjoint(wb, ref["psi_hat"]).real
        assert _rel(x.grad[b].cpu().numpy(), gwant) <= TOL16


def test_config4_iht_512_k49():
    """Inpainting at 512 x 512 with 49 filters (10 iterations): PSNR parity."""
    from paper_2006_04591_gb300 import apps
    ref, bank = _bank(512, 4)
    clean, mask, masked = synth.inpaint_batch(1, 512, 0.5, seed0=2000)
    out = apps.iht_inpaint(bank, torch.from_numpy(masked.astype(np.float32)).cuda(),
                           torch.from_numpy(mask.astype(np.float32)).cuda(), 10, 0.02)
    want = OA.iht_inpaint(masked[0].astype(np.float32).astype(np.float64), mask[0], ref["psi_hat"],
                          ref["rms"], 10, 0.02)
    p_gpu, p_ref = OA.psnr(clean[0], out.cpu().numpy()[0]), OA.psnr(clean[0], want)
    assert abs(p_gpu - p_ref) < 0.05, (p_gpu, p_ref)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_config5_1024_k49_batch8(dtype):
    """1024 x 1024, 49 filters, batch 8 in one call: sampled subbands of the
    decomposition and sampled images of the reconstruction vs the oracle."""
    ref, bank = _bank(1024, 4)
    x = np.stack([synth.cartoon(1024, 1024, 5000 + b) for b in range(8)]).astype(np.float32)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    tol = TOL32 if dtype == "f32" else TOL16
    c = bank.decompose(torch.from_numpy(x).cuda(), dtype=tdt)
    rng = np.random.default_rng(9)
    for _ in range(3):
        b, i = int(rng.integers(8)), int(rng.integers(49))
        want = OT.decompose(x[b], ref["psi_hat"][i:i + 1]).real[0]
        assert _rel(c[b, i].float().cpu().numpy(), want) <= tol, (b, i)
    r = bank.reconstruct(c)
    b = 7
    want = OT.reconstruct(c[b].float().cpu().numpy().astype(np.float64), ref["psi_hat"]).real
    assert _rel(r[b].cpu().numpy(), want) <= TOL32
