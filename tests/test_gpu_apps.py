"""Denoising (Sec. 4.2) and IHT inpainting (Sec. 4.3) on the GPU against the
FP64 oracle.  Hard thresholds are discontinuous, so parity is statistical:
PSNR within 0.05 dB, and for denoising the fraction of coefficients whose
keep/zero decision differs stays below 1e-4."""

import numpy as np
import pytest

from oracle import apps as OA
from oracle import bank as Bk
from oracle import transform as OT
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_denoise_matches_oracle():
    from paper_2006_04591_gb300 import apps
    from paper_2006_04591_gb300.shearlet import Bank
    N, sigma = 256, 30 / 255
    ref = Bk.shearlet_bank(N, N, 3)
    bank = Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    clean, noisy = synth.denoise_batch(2, N, sigma, seed0=100)
    xt = torch.from_numpy(noisy.astype(np.float32)).cuda()
    den = apps.denoise(bank, xt, sigma, 3.0).cpu().numpy()
    d = OA.subband_thresholds(ref["rms"], ref["idx"], sigma, 3.0)
    for b in range(2):
        want = OA.denoise(noisy[b].astype(np.float32).astype(np.float64), ref["psi_hat"], d)
        p_gpu, p_ref = OA.psnr(clean[b], den[b]), OA.psnr(clean[b], want)
        assert abs(p_gpu - p_ref) < 0.05, (p_gpu, p_ref)
        assert p_gpu > OA.psnr(clean[b], noisy[b]) + 5.0
        # decisions: GPU coefficients vs oracle coefficients against the same thresholds
        c_gpu = bank.decompose(xt[b:b + 1]).cpu().numpy()[0]
        c_ref = OT.decompose(noisy[b].astype(np.float32).astype(np.float64), ref["psi_hat"]).real
        th = d.astype(np.float32)[:, None, None]
        flips = np.mean((np.abs(c_gpu) >= th) != (np.abs(c_ref) >= th))
        assert flips < 1e-4


@pytest.mark.parametrize("kind", ["random", "squared"])
def test_iht_inpainting_matches_oracle(kind):
    """Both mask patterns of the inpainting experiments (Sec. 4.3)."""
    from paper_2006_04591_gb300 import apps
    from paper_2006_04591_gb300.shearlet import Bank
    N, T = 128, 20
    ref = Bk.shearlet_bank(N, N, 3)
    bank = Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    clean, mask, masked = synth.inpaint_batch(2, N, 0.5, seed0=2000, kind=kind)
    fm = torch.from_numpy(masked.astype(np.float32)).cuda()
    mk = torch.from_numpy(mask.astype(np.float32)).cuda()
    d0_gpu = apps.iht_start_threshold(bank, fm).cpu().numpy()
    out = apps.iht_inpaint(bank, fm, mk, T, 0.02).cpu().numpy()
    for b in range(2):
        want, hist, d0 = OA.iht_inpaint(masked[b].astype(np.float32).astype(np.float64), mask[b],
                                        ref["psi_hat"], ref["rms"], T, 0.02, return_history=True)
        assert abs(d0_gpu[b] - d0) <= 1e-5 * d0
        p_gpu, p_ref = OA.psnr(clean[b], out[b]), OA.psnr(clean[b], want)
        assert abs(p_gpu - p_ref) < 0.05, (p_gpu, p_ref)
        assert p_gpu > OA.psnr(clean[b], masked[b]) + (8.0 if kind == "random" else 2.0)


def test_iht_threshold_schedule_on_device():
    """shl_iht_thresholds against the oracle's schedule delta_t RMS_i
    (delta_0 = max |c_i| / RMS_i of SH f_masked, lambda reaching delta_min at
    the last iteration): the same start value and decay, no host round trip."""
    from paper_2006_04591_gb300 import apps
    from paper_2006_04591_gb300.shearlet import Bank
    N, T = 128, 12
    ref = Bk.shearlet_bank(N, N, 3)
    bank = Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    clean, mask, masked = synth.inpaint_batch(3, N, 0.5, seed0=2100)
    fm = torch.from_numpy(masked.astype(np.float32)).cuda()
    th = apps.iht_schedule(bank, fm, T, 0.02).cpu().numpy()          # [T, B, K]
    assert th.shape == (T, 3, bank.K)
    for b in range(3):
        _, hist, d0 = OA.iht_inpaint(masked[b].astype(np.float32).astype(np.float64), mask[b],
                                     ref["psi_hat"], ref["rms"], T, 0.02, return_history=True)
        want = hist[:, None] * ref["rms"][None, :]
        np.testing.assert_allclose(th[:, b, :], want, rtol=2e-5)
        np.testing.assert_allclose(th[-1, b, :], 0.02 * ref["rms"], rtol=2e-5)
    # a given start value: the same schedule for every image; one iteration
    th1 = apps.iht_schedule(bank, fm, 5, 0.1, delta_init=2.0).cpu().numpy()
    lam = (0.1 / 2.0) ** 0.25
    want1 = 2.0 * lam ** np.arange(5)[:, None, None] * ref["rms"][None, None, :]
    np.testing.assert_allclose(th1, np.broadcast_to(want1, th1.shape), rtol=1e-6)
    th0 = apps.iht_schedule(bank, fm, 1, 0.1, delta_init=3.0).cpu().numpy()
    np.testing.assert_allclose(th0[0], np.broadcast_to(3.0 * ref["rms"], (3, bank.K)), rtol=1e-6)
