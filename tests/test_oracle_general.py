"""Pins for the oracle at the sizes and spectra of the general kernels (CPU).

The general CUDA path computes the natural-order form c_i = ifft2(fft2(f)
G_i) on full complex planes for any size and for complex Hermitian spectra.
These checks tie that form to the paper's literal one (Sec. 3.3 shifts,
Sec. 3.4 listings) at odd, non-power-of-two and degenerate sizes, and check
the oracle's filter bank (Sec. 2.1, Eq. 3.2) at such sizes against the
properties the construction guarantees.
"""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as T

RNG = np.random.default_rng(2024)

SHAPES = [(9, 7), (5, 12), (15, 15), (1, 8), (3, 1), (1, 1), (27, 10)]


def _rand_complex(shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _hermitian_bank(K, N, M, rng=RNG):
    """Spectra of real, non-symmetric spatial filters: complex and Hermitian,
    G(-k) = conj(G(k)), in natural order."""
    g = rng.standard_normal((K, N, M))
    return np.fft.fft2(g, axes=(-2, -1))


@pytest.mark.parametrize("shape", SHAPES)
def test_natural_order_form_equals_literal_at_any_size(shape):
    N, M = shape
    psi_hat = np.stack([T.fourier(T.tfftshift(p)) for p in _rand_complex((3, N, M))])
    f = RNG.standard_normal((N, M))
    G = T.centred_to_natural(psi_hat)
    np.testing.assert_allclose(T.decompose_natural(f, G), T.decompose(f, psi_hat), rtol=0,
                               atol=1e-12 * np.abs(T.decompose(f, psi_hat)).max())
    c = _rand_complex((3, N, M))
    ref = T.reconstruct(c, psi_hat)
    np.testing.assert_allclose(T.reconstruct_natural(c, G), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())
    ref = T.adjoint(c, psi_hat)
    np.testing.assert_allclose(T.reconstruct_natural(c, G, weights=False), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(9, 7), (15, 15), (6, 10)])
def test_natural_form_is_spatial_correlation(shape):
    # Def. 2.6 sampled on the grid: c(m) = sum_n f(n + m) conj(psi(n)), with
    # the natural-order multiplier G = DFT of conj(psi) at negated frequency.
    N, M = shape
    psi = RNG.standard_normal((N, M))          # real, non-symmetric filter
    f = RNG.standard_normal((N, M))
    # sum_n f(n + m) psi(n) = ifft2(fft2(f) * conj(fft2(psi)))  (real psi)
    G = np.conj(np.fft.fft2(psi))[None]
    c = T.decompose_natural(f, G)[0]
    ref = T.correlate_direct(f, psi)
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(9, 7), (12, 5), (1, 6)])
def test_hermitian_spectra_give_real_coefficients_and_inverse(shape):
    N, M = shape
    G = _hermitian_bank(4, N, M)
    f = RNG.standard_normal((N, M))
    c = T.decompose_natural(f, G)
    assert np.abs(c.imag).max() < 1e-13 * np.abs(c.real).max()
    rec = T.reconstruct_natural(c.real, G)
    assert np.abs(rec.imag).max() < 1e-12
    np.testing.assert_allclose(rec.real, f, rtol=0, atol=1e-12 * np.abs(f).max())
    # adjointness on real data: <dec f, c> = <f, adj c>
    cc = RNG.standard_normal((4, N, M))
    lhs = np.sum(c.real * cc)
    rhs = np.sum(f * T.reconstruct_natural(cc, G, weights=False).real)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("rows,cols,J", [(45, 60, 2), (33, 33, 1), (100, 72, 2), (31, 17, 2)])
def test_bank_at_general_sizes(rows, cols, J):
    b = Bk.shearlet_bank(rows, cols, J)
    S = b["spectra"]
    assert S.shape == (Bk.n_shearlets(Bk.default_shear_levels(J)), rows, cols)
    neg = np.roll(np.roll(S[:, ::-1, ::-1], 1, axis=1), 1, axis=2)   # G(-k)
    assert np.abs(S - neg).max() == 0.0          # exactly even: real spatial filters
    assert b["dual_w"].min() > 0.0
    np.testing.assert_allclose(b["rms"] ** 2, np.sum(S ** 2, axis=(1, 2)) / (rows * cols))
    # the low-pass passes DC with gain 1 (H_J(0) = 1) and every band-pass blocks it
    assert abs(S[0, 0, 0] - 1.0) < 1e-12
    assert np.abs(S[1:, 0, 0]).max() < 1e-12
