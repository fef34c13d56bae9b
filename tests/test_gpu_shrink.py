"""shl_shrink, the fused denoise / IHT step (Sec. 4.2, 4.3): its row pass
thresholds each coefficient tile in registers, so it must give exactly the
bits of shl_decompose (float32) + shl_reconstruct(thresh) -- the same float32
values reach the same compare and the same transforms -- and match the FP64
oracle's threshold pipeline."""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import apps as OA
from oracle import bank as Bk
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_BANKS = {}


def _bank(rows, cols, J):
    key = (rows, cols, J)
    if key not in _BANKS:
        from paper_2006_04591_gb300.shearlet import Bank
        ref = Bk.shearlet_bank(rows, cols, J)
        _BANKS[key] = (ref, Bank.from_spectra(ref["spectra"], ref["idx"], device=0))
    return _BANKS[key]


def _inputs(B, rows, cols, K, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([synth.cartoon(rows, cols, seed + b) for b in range(B)]).astype(np.float32)
    x += rng.normal(0, 0.1, x.shape).astype(np.float32)
    th = rng.uniform(0.0, 0.15, (B, K)).astype(np.float32)
    th[:, 0] = 0.0
    return x, th


@pytest.mark.parametrize("rows,cols,J,B", [(16, 16, 1, 2), (64, 32, 2, 3), (256, 256, 3, 2),
                                           (512, 512, 4, 3), (32, 2048, 2, 1), (2048, 32, 2, 1)])
def test_shrink_equals_unfused_bits(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    x, th = _inputs(B, rows, cols, bank.K, rows + cols)
    xt, tht = torch.from_numpy(x).cuda(), torch.from_numpy(th).cuda()
    want = bank.reconstruct(bank.decompose(xt), thresh=tht)
    got = bank.shrink(xt, tht)
    assert torch.equal(got, want)


def test_masked_shrink_equals_unfused_and_aliases():
    ref, bank = _bank(256, 256, 3)
    B = 2
    x, th = _inputs(B, 256, 256, bank.K, 7)
    f = np.stack([synth.cartoon(256, 256, 70 + b) for b in range(B)]).astype(np.float32)
    m = np.stack([synth.bernoulli_mask(256, 256, 0.5, 80 + b) for b in range(B)]).astype(np.uint8)
    xt, tht, ft, mt = (torch.from_numpy(a).cuda() for a in (x, th, f, m))
    want = bank.reconstruct(bank.decompose_masked(xt, mt, ft), thresh=tht)
    got = bank.shrink(xt, tht, mask_u8=mt, f_est=ft)
    assert torch.equal(got, want)
    f2 = ft.clone()
    bank.shrink(xt, tht, mask_u8=mt, f_est=f2, out=f2)        # x_out aliases f_est
    assert torch.equal(f2, want)
    x2 = xt.clone()
    bank.shrink(x2, tht, out=x2)                               # x_out aliases x
    assert torch.equal(x2, bank.reconstruct(bank.decompose(xt), thresh=tht))


def test_shrink_zero_threshold_is_perfect_reconstruction_and_empty_batch():
    ref, bank = _bank(128, 128, 3)
    x, _ = _inputs(2, 128, 128, bank.K, 3)
    xt = torch.from_numpy(x).cuda()
    y = bank.shrink(xt, torch.zeros((2, bank.K), device="cuda"))
    assert (y - xt).abs().max().item() <= 1e-5 * xt.abs().max().item()
    e = bank.shrink(torch.empty((0, 128, 128), device="cuda"), torch.empty((0, bank.K), device="cuda"))
    assert e.shape == (0, 128, 128)


def test_shrink_denoise_matches_oracle_psnr():
    sigma = 30 / 255
    ref, bank = _bank(512, 512, 4)
    clean, noisy = synth.denoise_batch(2, 512, sigma, seed0=300)
    d = OA.subband_thresholds(ref["rms"], ref["idx"], sigma, 3.0)
    th = torch.from_numpy(np.tile(d.astype(np.float32), (2, 1))).cuda()
    den = bank.shrink(torch.from_numpy(noisy.astype(np.float32)).cuda(), th).cpu().numpy()
    for b in range(2):
        want = OA.denoise(noisy[b].astype(np.float32).astype(np.float64), ref["psi_hat"], d)
        assert abs(OA.psnr(clean[b], den[b]) - OA.psnr(clean[b], want)) < 0.05


CHUNKED = textwrap.dedent("""
    import numpy as np, torch
    from oracle import bank as Bk
    from paper_2006_04591_gb300 import shearlet as S
    from paper_2006_04591_gb300 import synth
    ref = Bk.shearlet_bank(512, 512, 2)
    bank = S.Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    rng = np.random.default_rng(5)
    x = np.stack([synth.cartoon(512, 512, 500 + b) for b in range(3)]).astype(np.float32)
    th = rng.uniform(0, 0.1, (3, bank.K)).astype(np.float32)
    xt, tht = torch.from_numpy(x).cuda(), torch.from_numpy(th).cuda()
    want = bank.reconstruct(bank.decompose(xt), thresh=tht)
    got = bank.shrink(xt, tht)
    assert torch.equal(got, want)
    z = bank.shrink(xt, torch.zeros_like(tht))
    assert (z - xt).abs().max().item() <= 1e-5 * xt.abs().max().item()
    print("chunked ok")
""")


def test_shrink_with_chunks_inside_an_image():
    """3 MB staging = 2 subband planes at 512 x 512, K = 17: the reconstruction
    sums carry partial spectra between chunks of one image."""
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    env["SHL_STAGE_MB"] = "3"
    r = subprocess.run([sys.executable, "-c", CHUNKED], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "chunked ok" in r.stdout
