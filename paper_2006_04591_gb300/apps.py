"""Shearlet denoising (Sec. 4.2) and inpainting by iterative hard thresholding
(Sec. 4.3, Alg. "Shearlet inpainting by iterative hard thresholding") on the
GPU through libshearlet.

Every transform, threshold and residual step runs in the library's kernels.
With float32 coefficients both loops call shl_shrink, which thresholds each
row tile of coefficients in registers between the decomposition's and the
reconstruction's row passes, so the coefficients never reach memory; with
bfloat16 coefficients (or fused=False) the decomposition stores them and the
reconstruction applies the threshold while reading them.  The inpainting
residual M (f_masked - f) + f is formed while the first pass reads its input.  Thresholds are per (image, subband):
  denoising   delta_i = factor_{scale(i)} * sigma * RMS_i, low-pass kept;
  inpainting  delta_t * RMS_i for every subband, delta_t = delta_init lambda^t,
              lambda = (delta_min / delta_init)^(1 / (T - 1)),
              delta_init = max_{i,n} |c_i(n)| / RMS_i of SH f_masked.
"""

from __future__ import annotations

import numpy as np
import torch

from .shearlet import SHL_OP_DECOMPOSE, SHL_OP_RECONSTRUCT, SHL_OP_SHRINK, Bank


def denoise_thresholds(bank: Bank, sigma: float, factors, batch: int) -> torch.Tensor:
    """[batch, K] thresholds factor_{scale} sigma RMS_i (0 for the low-pass)."""
    th = np.zeros(bank.K, np.float32)
    for i, (cone, scale, _k) in enumerate(bank.idx):
        if cone == 0:
            continue
        f = factors if np.isscalar(factors) else factors[scale - 1]
        th[i] = f * sigma * bank.rms[i]
    return torch.from_numpy(np.tile(th, (batch, 1))).cuda(bank.device)


def denoise(bank: Bank, x_noisy: torch.Tensor, sigma: float, factors=3.0,
            coeff_dtype=torch.float32, fused=True, ws=None) -> torch.Tensor:
    """SH^{-1} T_delta SH x for a batch [B, N, M] (float32)."""
    B = x_noisy.shape[0]
    th = denoise_thresholds(bank, sigma, factors, B)
    if fused and coeff_dtype == torch.float32:
        return bank.shrink(x_noisy, th, ws=ws)
    c = bank.decompose(x_noisy, dtype=coeff_dtype)
    return bank.reconstruct(c, thresh=th)


def iht_start_threshold(bank: Bank, f_masked: torch.Tensor, coeffs=None) -> torch.Tensor:
    """delta_init per image: max_{i,n} |c_i(n)| / RMS_i of SH f_masked ([B])."""
    return iht_start_absmax(bank, f_masked, coeffs).amax(dim=1)


def iht_start_absmax(bank: Bank, f_masked: torch.Tensor, coeffs=None) -> torch.Tensor:
    """max_n |c_i(n)| / RMS_i of SH f_masked per (image, subband), [B, K] on the device."""
    c = bank.decompose(f_masked, out=coeffs)
    return bank.subband_absmax(c, by_rms=True)


def iht_schedule(bank: Bank, f_masked: torch.Tensor, iterations: int, delta_min: float = 0.02,
                 delta_init=None, coeffs=None) -> torch.Tensor:
    """Thresholds delta_t RMS_i of every iteration, [T, B, K], formed on the
    device (shl_iht_thresholds): no host read between the start value and
    the loop.  delta_init None: max_{i,n} |c_i(n)| / RMS_i of SH f_masked."""
    B = f_masked.shape[0]
    if delta_init is None:
        a = iht_start_absmax(bank, f_masked, coeffs)
    else:
        d = torch.as_tensor(delta_init, dtype=torch.float32).to(f_masked.device).reshape(-1)
        a = d.expand(B).reshape(B, 1).expand(B, bank.K).contiguous()
    return bank.iht_thresholds(a, iterations, delta_min)


def iht_inpaint(bank: Bank, f_masked: torch.Tensor, mask: torch.Tensor, iterations: int,
                delta_min: float = 0.02, delta_init=None, coeff_dtype=torch.float32,
                f_init=None, fused=True):
    """Alg. "Shearlet inpainting by iterative hard thresholding" for a batch.

    f_masked: [B, N, M] float32; mask: [B, N, M] (nonzero = observed).
    Returns the inpainted batch (float32).
    """
    B = f_masked.shape[0]
    dev = f_masked.device
    mask_u8 = (mask != 0).to(torch.uint8).contiguous()
    f_masked = f_masked.contiguous().float()
    fused = fused and coeff_dtype == torch.float32
    coeffs = None
    if delta_init is None or not fused:
        coeffs = torch.empty((B, bank.K, bank.rows, bank.cols), dtype=coeff_dtype, device=dev)
    T = iterations
    th = iht_schedule(bank, f_masked, T, delta_min, delta_init, coeffs)   # [T, B, K], device
    f = torch.zeros_like(f_masked) if f_init is None else f_init.contiguous().float().clone()
    g = torch.empty_like(f)
    if fused:
        ws = bank.workspace(SHL_OP_SHRINK, B)
        for t in range(T):
            bank.shrink(f_masked, th[t], mask_u8=mask_u8, f_est=f, out=g, ws=ws)
            f, g = g, f
        return f
    ws_d = bank.workspace(SHL_OP_DECOMPOSE, B)
    ws_r = bank.workspace(SHL_OP_RECONSTRUCT, B)
    for t in range(T):
        bank.decompose_masked(f_masked, mask_u8, f, out=coeffs, ws=ws_d)
        bank.reconstruct(coeffs, thresh=th[t], out=g, ws=ws_r)
        f, g = g, f
    return f


def psnr(a: torch.Tensor, b: torch.Tensor, peak: float = 1.0) -> torch.Tensor:
    """Per-image PSNR (Sec. 4.2): 20 log10(peak sqrt(Npix) / ||a - b||_F)."""
    err = (a.double() - b.double()).flatten(1).norm(dim=1)
    n = a[0].numel()
    return 20.0 * torch.log10(peak * (n ** 0.5) / err)
