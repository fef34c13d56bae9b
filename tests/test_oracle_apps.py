"""Pins for the oracle's applications (CPU only): threshold, PSNR, denoise, IHT."""

import numpy as np

from oracle import apps as A
from oracle import bank as Bk
from oracle import transform as T


def test_hard_threshold_keeps_ties():
    x = np.array([-2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0])
    np.testing.assert_array_equal(A.hard_threshold(x, 1.0), [-2, -1, 0, 0, 0, 1, 2])


def test_psnr_closed_form():
    f = np.zeros((8, 8))
    g = np.full((8, 8), 0.1)
    assert abs(A.psnr(f, g) - 20.0) < 1e-12
    # 255-scaled images give the same number with peak 255 (Sec. 4.2 formula)
    assert abs(A.psnr(255 * f, 255 * g, peak=255.0) - 20.0) < 1e-12


def test_thresholds_skip_lowpass_and_scale_by_rms():
    b = Bk.shearlet_bank(32, 32, 2)
    d = A.subband_thresholds(b["rms"], b["idx"], 0.1, [2.0, 3.0])
    assert d[0] == 0.0
    for i in range(1, len(d)):
        f = 2.0 if b["idx"][i][1] == 1 else 3.0
        assert abs(d[i] - f * 0.1 * b["rms"][i]) < 1e-15


def test_denoise_with_zero_thresholds_is_identity():
    b = Bk.shearlet_bank(32, 32, 2)
    f = np.random.default_rng(0).standard_normal((32, 32))
    out = A.denoise(f, b["psi_hat"], np.zeros(len(b["rms"])))
    np.testing.assert_allclose(out, f, atol=1e-12)


def test_iht_schedule_and_limits():
    b = Bk.shearlet_bank(32, 32, 2)
    rng = np.random.default_rng(1)
    f = rng.uniform(size=(32, 32))
    ones = np.ones_like(f)
    out, hist, d0 = A.iht_inpaint(f, ones, b["psi_hat"], b["rms"], 5, 0.02,
                                  return_history=True)
    assert abs(hist[0] - d0) < 1e-15 and abs(hist[-1] - 0.02) < 1e-12
    np.testing.assert_allclose(hist[1:] / hist[:-1], (0.02 / d0) ** 0.25, rtol=1e-12)
    # full mask, vanishing threshold: one iteration reproduces the image
    out = A.iht_inpaint(f, ones, b["psi_hat"], b["rms"], 1, delta_init=0.0)
    np.testing.assert_allclose(out, f, atol=1e-12)
    # empty mask: nothing is ever observed, the estimate stays zero
    out = A.iht_inpaint(f * 0, ones * 0, b["psi_hat"], b["rms"], 3, delta_init=1.0)
    assert np.abs(out).max() == 0.0


def test_iht_improves_masked_image():
    from paper_2006_04591_gb300 import synth
    N = 64
    b = Bk.shearlet_bank(N, N, 3)
    clean = synth.cartoon(N, N, seed=3)
    mask = synth.bernoulli_mask(N, N, 0.5, seed=4)
    out = A.iht_inpaint(clean * mask, mask, b["psi_hat"], b["rms"], 20)
    assert A.psnr(clean, out) > A.psnr(clean, clean * mask) + 8.0
