"""GPU parity of the general kernels (any size 1..4096, complex Hermitian
spectra) against the FP64 oracle, element by element.

The oracle side is the natural-order form c_i = ifft2(fft2(f) G_i) and its
reconstruction / adjoint, which ``tests/test_oracle_general.py`` ties to the
paper's literal shifted form at these sizes.  Banks are the oracle's
shearlet system at general sizes, spectra of random real filters (complex,
Hermitian) and random even real spectra for the degenerate sizes; none of
them comes from the CUDA path.  Error measure: max |gpu - oracle| / max
|oracle| per image (float32 <= 1e-5, bfloat16-stored coefficients <= 1e-2).
"""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as T
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL32 = 1e-5
TOL16 = 1e-2

# (kind, rows, cols, J or K, batch).  127, 131, 257 and 4093 are primes above
# the largest direct radix (Bluestein lines); 8 x 16 is a power of two below
# the half-spectrum kernels' range; 1 x 1, 1 x 37 and 3 x 1 are degenerate.
CASES = [
    ("shear", 45, 60, 2, 3), ("shear", 33, 33, 1, 2), ("shear", 127, 128, 2, 2),
    ("shear", 100, 72, 2, 2), ("shear", 8, 16, 1, 2), ("shear", 240, 320, 3, 2),
    ("herm", 9, 7, 4, 3), ("herm", 64, 50, 5, 2), ("herm", 131, 20, 3, 2),
    ("herm", 20, 257, 3, 1),
    ("even", 1, 1, 2, 2), ("even", 1, 37, 3, 2), ("even", 3, 1, 2, 2),
]
MAX_CASES = [("herm", 4093, 17, 2, 1), ("even", 17, 4093, 2, 1), ("even", 4096, 24, 2, 1)]
_BANKS = {}


def _spectra(kind, rows, cols, n, seed=5):
    """Natural-order spectra [K, rows, cols] (and idx) of one test bank.

    The random banks get one more, real and even, filter sqrt(1.1 max W' - W')
    (W' the dual weights of the random filters), which makes W constant: as
    well conditioned as a tight frame, so 1/W does not amplify rounding."""
    rng = np.random.default_rng(seed + rows * 7 + cols)
    if kind == "shear":
        ref = Bk.shearlet_bank(rows, cols, n)
        return ref["spectra"], ref["idx"]
    g = rng.standard_normal((n, rows, cols))
    if kind == "herm":        # real, non-symmetric filters: complex Hermitian spectra
        G = np.fft.fft2(g, axes=(-2, -1)) / np.sqrt(rows * cols)
    else:                     # point-symmetric real filters: real, even spectra
        g = 0.5 * (g + np.roll(np.roll(g[:, ::-1, ::-1], 1, axis=1), 1, axis=2))
        G = np.fft.fft2(g, axes=(-2, -1)).real / np.sqrt(rows * cols)
    Wp = np.sum(np.abs(G) ** 2, axis=0)
    fill = np.sqrt(1.1 * Wp.max() - Wp)[None]
    return np.concatenate([G, fill.astype(G.dtype)]), None


def _bank(kind, rows, cols, n):
    key = (kind, rows, cols, n)
    if key not in _BANKS:
        from paper_2006_04591_gb300.shearlet import Bank
        G, idx = _spectra(kind, rows, cols, n)
        b = Bank.from_complex_spectra(G, idx, device=0) if kind == "herm" else \
            Bank.from_spectra(G, idx, device=0)
        assert b.general
        _BANKS[key] = (G, b)
    return _BANKS[key]


def _images(B, rows, cols, seed):
    return np.stack([synth.cartoon(rows, cols, seed + b) +
                     synth.gaussian_noise((rows, cols), 0.05, 900 + seed + b)
                     for b in range(B)]).astype(np.float32)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _dec64(x, G, dual=False):
    W = np.sum(np.abs(G) ** 2, axis=0)
    Gd = G / W if dual else G
    out = np.stack([T.decompose_natural(xb, Gd) for xb in np.asarray(x, np.float64)])
    assert np.abs(out.imag).max() <= 1e-9 * max(np.abs(out.real).max(), 1e-300)
    return out.real


def _rec64(c, G, weights=True):
    out = np.stack([T.reconstruct_natural(cb, G, weights) for cb in np.asarray(c, np.float64)])
    return out.real


def _per_image(got, want, tol):
    for b in range(want.shape[0]):
        assert _rel(got[b], want[b]) <= tol, (b, _rel(got[b], want[b]))


@pytest.mark.parametrize("kind,rows,cols,n,B", CASES + MAX_CASES)
def test_decompose_and_reconstruct(kind, rows, cols, n, B):
    G, bank = _bank(kind, rows, cols, n)
    x = _images(B, rows, cols, 11)
    xt = torch.from_numpy(x).cuda()
    c = bank.decompose(xt)
    want = _dec64(x, G)
    _per_image(c.cpu().numpy(), want, TOL32)
    cc = np.random.default_rng(3).standard_normal(c.shape).astype(np.float32)
    ct = torch.from_numpy(cc).cuda()
    _per_image(bank.reconstruct(ct).cpu().numpy(), _rec64(cc, G), TOL32)
    _per_image(bank.adjoint(ct).cpu().numpy(), _rec64(cc, G, weights=False), TOL32)
    # perfect reconstruction through the GPU path
    y = bank.reconstruct(c).cpu().numpy()
    assert _rel(y, x) <= TOL32 * 4


@pytest.mark.parametrize("kind,rows,cols,n,B", CASES[:10])
def test_dual_weighted_and_bf16(kind, rows, cols, n, B):
    G, bank = _bank(kind, rows, cols, n)
    x = _images(B, rows, cols, 21)
    xt = torch.from_numpy(x).cuda()
    _per_image(bank.decompose(xt, dual=True).cpu().numpy(), _dec64(x, G, dual=True), TOL32)
    c16 = bank.decompose(xt, dtype=torch.bfloat16)
    _per_image(c16.float().cpu().numpy(), _dec64(x, G), TOL16)
    # bfloat16 coefficients in: the oracle reconstructs the same rounded values
    c16f = c16.float().cpu().numpy()
    _per_image(bank.reconstruct(c16).cpu().numpy(), _rec64(c16f, G), TOL32)


@pytest.mark.parametrize("kind,rows,cols,n,B", [CASES[0], CASES[2], CASES[6], CASES[8]])
def test_threshold_on_read_and_masked_input(kind, rows, cols, n, B):
    G, bank = _bank(kind, rows, cols, n)
    rng = np.random.default_rng(9)
    c = rng.standard_normal((B, bank.K, rows, cols)).astype(np.float32)
    th = rng.uniform(0.0, 1.5, (B, bank.K)).astype(np.float32)
    ct, tht = torch.from_numpy(c).cuda(), torch.from_numpy(th).cuda()
    kept = np.where(np.abs(c) >= th[:, :, None, None], c, 0.0)   # same float32 compare
    _per_image(bank.reconstruct(ct, thresh=tht).cpu().numpy(), _rec64(kept, G), TOL32)
    fm = _images(B, rows, cols, 31)
    fe = _images(B, rows, cols, 41)
    m = np.stack([synth.bernoulli_mask(rows, cols, 0.5, 50 + b) for b in range(B)]).astype(np.uint8)
    u = np.where(m != 0, fm, fe)
    got = bank.decompose_masked(*(torch.from_numpy(a).cuda() for a in (fm, m, fe)))
    _per_image(got.cpu().numpy(), _dec64(u, G), TOL32)


def _safe_thresholds(c64, rng, margin=1e-4):
    """Per-subband thresholds that sit in a gap of the oracle's |c|, at least
    margin * max|c| from every coefficient, so that float32 rounding of the
    GPU's coefficients cannot flip a keep / zero decision."""
    B, K = c64.shape[:2]
    th = np.zeros((B, K), np.float32)
    for b in range(B):
        scale = np.abs(c64[b]).max()
        for i in range(K):
            a = np.sort(np.abs(c64[b, i]).ravel())
            lo = a.size // 4
            gaps = np.nonzero(np.diff(a[lo:]) > 2 * margin * scale)[0]
            if gaps.size:
                j = lo + gaps[rng.integers(gaps.size)]
                th[b, i] = 0.5 * (a[j] + a[j + 1])
            else:
                th[b, i] = 2.0 * a[-1] + 1.0       # zero the whole subband
            assert np.abs(np.abs(c64[b, i]) - th[b, i]).min() > margin * scale
    return th


@pytest.mark.parametrize("kind,rows,cols,n,B", [CASES[0], CASES[2], CASES[7], CASES[11]])
def test_shrink_matches_oracle_and_unfused(kind, rows, cols, n, B):
    G, bank = _bank(kind, rows, cols, n)
    x = _images(B, rows, cols, 61)
    c64 = _dec64(x, G)
    th = _safe_thresholds(c64, np.random.default_rng(1))
    want = _rec64(np.where(np.abs(c64) >= th[:, :, None, None], c64, 0.0), G)
    xt, tht = torch.from_numpy(x).cuda(), torch.from_numpy(th).cuda()
    got = bank.shrink(xt, tht)
    _per_image(got.cpu().numpy(), want, TOL32 * 4)
    assert torch.equal(got, bank.reconstruct(bank.decompose(xt), thresh=tht))
    m = np.stack([synth.bernoulli_mask(rows, cols, 0.5, 70 + b) for b in range(B)]).astype(np.uint8)
    fe = _images(B, rows, cols, 81)
    mt, fet = torch.from_numpy(m).cuda(), torch.from_numpy(fe).cuda()
    assert torch.equal(bank.shrink(xt, tht, mask_u8=mt, f_est=fet),
                       bank.reconstruct(bank.decompose_masked(xt, mt, fet), thresh=tht))


def test_general_path_agrees_with_half_spectrum_path():
    from paper_2006_04591_gb300.shearlet import Bank
    ref = Bk.shearlet_bank(64, 128, 3)
    fast = Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    gen = Bank.from_complex_spectra(ref["spectra"], ref["idx"], device=0)
    assert not fast.general and gen.general
    x = torch.from_numpy(_images(3, 64, 128, 5)).cuda()
    a, b = fast.decompose(x), gen.decompose(x)
    assert (a - b).abs().max().item() <= 2e-6 * a.abs().max().item()
    assert (fast.reconstruct(a) - gen.reconstruct(a)).abs().max().item() <= 2e-6 * x.abs().max().item()


def test_large_plane_parity():
    # 1000 x 1500 (radices 4 4 4 ... 5 5 5 3): sampled subbands against the oracle
    G, bank = _bank("shear", 1000, 1500, 2)
    x = _images(1, 1000, 1500, 91)
    xt = torch.from_numpy(x).cuda()
    c = bank.decompose(xt)
    for i in (0, 5, 16):
        want = T.decompose_natural(x[0].astype(np.float64), G[i:i + 1])[0].real
        assert _rel(c[0, i].cpu().numpy(), want) <= TOL32
    assert _rel(bank.reconstruct(c).cpu().numpy(), x) <= TOL32 * 4


def test_absmax_and_empty_batch():
    G, bank = _bank("herm", 64, 50, 5)
    x = torch.from_numpy(_images(2, 64, 50, 3)).cuda()
    c = bank.decompose(x)
    m = bank.subband_absmax(c)
    assert torch.equal(m, c.abs().amax(dim=(2, 3)))
    e = bank.decompose(torch.empty((0, 64, 50), device="cuda"))
    assert e.shape == (0, bank.K, 64, 50)
    r = bank.reconstruct(torch.empty((0, bank.K, 64, 50), device="cuda"))
    assert r.shape == (0, 64, 50)


def test_chunked_staging_with_partial_sums():
    """A staging area of two planes splits each image's 17 filters over 9
    chunks, so the reconstruction carries partial sums between launches."""
    script = textwrap.dedent("""
        import numpy as np, torch, sys
        sys.path.insert(0, %r)
        from oracle import bank as Bk, transform as T
        from paper_2006_04591_gb300.shearlet import Bank
        from paper_2006_04591_gb300 import synth
        ref = Bk.shearlet_bank(45, 60, 2)
        G = ref["spectra"]
        bank = Bank.from_spectra(G, ref["idx"], device=0)
        x = np.stack([synth.cartoon(45, 60, s) for s in (1, 2, 3)]).astype(np.float32)
        xt = torch.from_numpy(x).cuda()
        c = bank.decompose(xt)
        want = np.stack([T.decompose_natural(xb.astype(np.float64), G).real for xb in x])
        e1 = np.abs(c.cpu().numpy() - want).max() / np.abs(want).max()
        y = bank.reconstruct(c)
        e2 = np.abs(y.cpu().numpy() - x).max() / np.abs(x).max()
        th = torch.full((3, bank.K), 0.01, device="cuda")
        same = torch.equal(bank.shrink(xt, th), bank.reconstruct(c, thresh=th))
        print(e1, e2, same)
        assert e1 <= 1e-5 and e2 <= 4e-5 and same
    """ % ROOT)
    env = dict(os.environ, SHL_STAGE_MB="0.045")    # 45 x 60 x 8 B = 21.6 KB per plane
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
