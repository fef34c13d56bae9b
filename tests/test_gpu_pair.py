"""GPU parity of the paired-subband kernels (one cluster launch per direction,
two subbands per complex plane) against the FP64 oracle.

These kernels are the opt-in path (SHL_FUSED=1, read once per process) for
square 512 x 512 planes; each test runs its checks in a child process with
the switch set and asserts, from the library's launch profile, that the
paired kernels ran.  Odd filter counts leave one subband of each image
without a partner (its imaginary half is zero), even counts pair every
subband; small batches give fewer pairs than co-resident clusters, the
16-image batch splits images across clusters, whose partial sums are added
in a fixed order.  Banks come from the oracle (shearlet systems, random real
even filters completed to a constant W); error measure max |gpu - oracle| /
max |oracle| per image (float32 <= 1e-5, bfloat16-stored coefficients
<= 1e-2).
"""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:            # the child process runs this file as a script
    sys.path.insert(0, ROOT)

from oracle import bank as Bk
from oracle import transform as OT
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 1e-2
N = 512
_BANKS = {}


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _even_spectra(K, seed):
    """K - 1 random point-symmetric real filters plus one real even filter
    that makes W constant (natural-order spectra)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((max(K - 1, 1), N, N))
    g = 0.5 * (g + np.roll(np.roll(g[:, ::-1, ::-1], 1, axis=1), 1, axis=2))
    G = np.fft.fft2(g, axes=(-2, -1)).real / N
    if K == 1:                          # one positive even filter
        return np.exp(0.3 * G)
    Wp = np.sum(G ** 2, axis=0)
    return np.concatenate([G, np.sqrt(1.1 * Wp.max() - Wp)[None]])


def _bank(kind, n):
    """('shear', J): the oracle's shearlet system; ('even', K): random bank."""
    key = (kind, n)
    if key not in _BANKS:
        from paper_2006_04591_gb300.shearlet import Bank
        if kind == "shear":
            ref = Bk.shearlet_bank(N, N, n)
            G = ref["spectra"]                  # natural order, real and even
            b = Bank.from_spectra(G, ref["idx"], device=0)
        else:
            G = _even_spectra(n, 40 + n)
            b = Bank.from_spectra(G, device=0)
        assert not b.general
        _BANKS[key] = (G, b)
    return _BANKS[key]


def _images(B, seed):
    return np.stack([synth.cartoon(N, N, seed + b) +
                     synth.gaussian_noise((N, N), 0.05, 900 + seed + b)
                     for b in range(B)]).astype(np.float32)


def _dec64(x, G, dual=False):
    W = np.sum(G ** 2, axis=0)
    Gd = G / W if dual else G
    return np.stack([OT.decompose_natural(xb, Gd).real for xb in np.asarray(x, np.float64)])


def _rec64(c, G, weights=True):
    return np.stack([OT.reconstruct_natural(cb, G, weights).real
                     for cb in np.asarray(c, np.float64)])


def _per_image(got, want, tol):
    for b in range(want.shape[0]):
        e = _rel(got[b], want[b])
        assert e <= tol, (b, e)


CASES = [("shear", 2, 1), ("shear", 3, 2), ("shear", 4, 3), ("even", 6, 2), ("even", 1, 2),
         ("even", 2, 1)]


def _case_decompose(kind, n, B):
    G, bank = _bank(kind, n)
    x = _images(B, 10 + n)
    xt = torch.from_numpy(x).cuda()
    want = _dec64(x, G)
    _per_image(bank.decompose(xt).cpu().numpy(), want, TOL32)
    _per_image(bank.decompose(xt, dtype=torch.bfloat16).float().cpu().numpy(), want, TOL16)
    _per_image(bank.decompose(xt, dual=True).cpu().numpy(), _dec64(x, G, dual=True), TOL32)


def _case_reconstruct(kind, n, B):
    G, bank = _bank(kind, n)
    K = G.shape[0]
    rng = np.random.default_rng(7 * n + B)
    c = rng.standard_normal((B, K, N, N)).astype(np.float32)
    ct = torch.from_numpy(c).cuda()
    _per_image(bank.reconstruct(ct).cpu().numpy(), _rec64(c, G), TOL32)
    _per_image(bank.adjoint(ct).cpu().numpy(), _rec64(c, G, weights=False), TOL32)
    th = rng.uniform(0, 1.5, size=(B, K)).astype(np.float32)
    th[0, 0] = 0.0
    kept = np.where(np.abs(c) >= th[:, :, None, None], c, 0.0)   # the same float32 compare
    got = bank.reconstruct(ct, thresh=torch.from_numpy(th).cuda()).cpu().numpy()
    _per_image(got, _rec64(kept, G), TOL32)
    c16 = ct.bfloat16()
    _per_image(bank.reconstruct(c16).cpu().numpy(), _rec64(c16.float().cpu().numpy(), G), TOL32)


def _case_round_trip():
    """Perfect reconstruction through both kernels, and the same bits on a
    second call (partial sums are combined in a fixed order)."""
    G, bank = _bank("shear", 4)
    x = torch.from_numpy(_images(5, 77)).cuda()
    c = bank.decompose(x)
    r = bank.reconstruct(c)
    assert (r - x).abs().max().item() <= TOL32 * x.abs().max().item()
    assert torch.equal(c, bank.decompose(x))
    assert torch.equal(r, bank.reconstruct(c))


def _case_adjoint_16():
    """<dec x, w> = <x, adj w> at the benchmark's batch (images split across
    clusters)."""
    G, bank = _bank("shear", 4)
    x = torch.from_numpy(_images(16, 300)).cuda()
    c = bank.decompose(x)
    w = torch.randn(c.shape, generator=torch.Generator().manual_seed(5)).cuda()
    a = bank.adjoint(w)
    lhs = (c.double() * w.double()).sum().item()
    rhs = (x.double() * a.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def _paired_kernels_ran():
    from paper_2006_04591_gb300 import shearlet as S
    prof = S.shl_profile_read()
    assert "pair_dec" in prof or "pair_rec" in prof, sorted(prof)


def _child(name, *args):
    """Run _case_<name>(*args) in a process with the paired kernels on."""
    env = dict(os.environ, SHL_FUSED="1")
    cmd = [sys.executable, os.path.abspath(__file__), name] + [str(a) for a in args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "paired ok" in r.stdout


@pytest.mark.parametrize("kind,n,B", CASES)
def test_pair_decompose_f32_bf16_dual(kind, n, B):
    _child("decompose", kind, n, B)


@pytest.mark.parametrize("kind,n,B", CASES)
def test_pair_reconstruct_adjoint_threshold(kind, n, B):
    _child("reconstruct", kind, n, B)


def test_pair_round_trip_and_repeatability():
    _child("round_trip")


def test_pair_adjoint_identity_16_images():
    _child("adjoint_16")


if __name__ == "__main__":
    from paper_2006_04591_gb300 import _build
    from paper_2006_04591_gb300 import shearlet as S
    _build.build()
    S.shl_profile_enable(1)
    name, rest = sys.argv[1], sys.argv[2:]
    args = [int(a) if a.lstrip("-").isdigit() else a for a in rest]
    globals()["_case_" + name](*args)
    torch.cuda.synchronize()
    _paired_kernels_ran()
    print("paired ok")
