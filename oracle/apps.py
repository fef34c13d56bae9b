"""FP64 oracle: thresholding, PSNR, denoising and IHT inpainting (Sec. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Hard thresholding (Sec. 4.2): keep x(n) when |x(n)| >= delta, else 0.  The
  tie |x| = delta is kept.
* PSNR (Sec. 4.2): ``20 log10(peak sqrt(Npix) / ||f - g||_F)`` with peak 255
  for 8-bit images; images in [0, 1] use peak 1, which is the same number.
* Denoising (Sec. 4.2): ``SH^{-1} T_delta SH f_noisy`` with per-subband
  thresholds ``factor_j * sigma * RMS_i`` (the listing multiplies the
  per-scale factor by each filter's RMS).  Reading: the low-pass subband is
  not thresholded (the paper's factors are per shearlet scale only).
* Inpainting (Alg. "Shearlet inpainting by iterative hard thresholding"):
  ``f_res = M (f_masked - f_inp)``;
  ``f_inp = SH^{-1} T_delta SH (f_res + f_inp)``; ``delta *= lambda``.
  Readings: lambda = (delta_min / delta_init)^{1/(T-1)} so that delta reaches
  delta_min on the last iteration (the printed lambda assumes
  delta_init = 1); delta is relative to each filter's RMS, i.e. subband i is
  thresholded at ``delta * RMS_i``, the low-pass included;
  ``delta_init = max_{i,n} |c_i(n)| / RMS_i`` of SH f_masked.
"""

from __future__ import annotations

import numpy as np

from . import transform as T


def hard_threshold(x: np.ndarray, delta) -> np.ndarray:
    """T_delta x: zero every entry with |x| < delta (ties kept)."""
    x = np.asarray(x)
    return np.where(np.abs(x) >= delta, x, 0.0)


def psnr(f: np.ndarray, g: np.ndarray, peak: float = 1.0) -> float:
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    err = np.linalg.norm((f - g).ravel())
    return float(20.0 * np.log10(peak * np.sqrt(f.size) / err))


def subband_thresholds(rms, idx, sigma: float, factors) -> np.ndarray:
    """delta_i = factor_{scale(i)} sigma RMS_i; 0 for the low-pass."""
    rms = np.asarray(rms, dtype=np.float64)
    idx = np.asarray(idx)
    out = np.zeros(len(rms))
    for i in range(len(rms)):
        cone, scale = int(idx[i][0]), int(idx[i][1])
        if cone == 0:
            continue
        f = factors if np.isscalar(factors) else factors[scale - 1]
        out[i] = f * sigma * rms[i]
    return out


def denoise(f_noisy: np.ndarray, psi_hat: np.ndarray, deltas) -> np.ndarray:
    """SH^{-1} T_delta SH f for one image; deltas [K] per subband."""
    c = T.decompose(f_noisy, psi_hat).real
    c = np.stack([hard_threshold(c[i], deltas[i]) for i in range(len(c))])
    return T.reconstruct(c, psi_hat).real


def iht_inpaint(f_masked: np.ndarray, mask: np.ndarray, psi_hat: np.ndarray,
                rms, iterations: int, delta_min: float = 0.02,
                delta_init=None, return_history: bool = False):
    """Alg. "Shearlet inpainting by iterative hard thresholding", one image."""
    rms = np.asarray(rms, dtype=np.float64)
    f_masked = np.asarray(f_masked, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    if delta_init is None:
        c0 = T.decompose(f_masked, psi_hat).real
        delta_init = float(np.max(np.abs(c0) / rms[:, None, None]))
    lam = (delta_min / delta_init) ** (1.0 / (iterations - 1)) if iterations > 1 else 1.0
    f_inp = np.zeros_like(f_masked)
    delta = delta_init
    hist = []
    for _ in range(iterations):
        f_res = mask * (f_masked - f_inp)
        c = T.decompose(f_res + f_inp, psi_hat).real
        c = np.stack([hard_threshold(c[i], delta * rms[i]) for i in range(len(c))])
        f_inp = T.reconstruct(c, psi_hat).real
        hist.append(delta)
        delta = lam * delta
    if return_history:
        return f_inp, np.asarray(hist), delta_init
    return f_inp
