"""Pins for the oracle's filter bank (CPU only).

The bank's parts are checked against their definitions computed another
way: filter design constraints from the taps, iterated filters from explicit
convolutions, the fan filter from its spatial polynomial, the digital shear
from a literal loop over Eqs. 2.4-2.5, the filter count of Eq. 3.2 under the
stated shear-level reading, and frame properties (real even spectra, W > 0,
RMS = spatial l2 norm, noise statistics).
"""

import math

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as T


def _dtft(taps, w):
    """DTFT of centred taps (index len//2 is n=0) at frequencies w."""
    n = np.arange(len(taps)) - (len(taps) - 1) // 2
    return np.sum(taps[None, :] * np.exp(-1j * np.outer(w, n)), axis=1)


def test_lowpass_design_constraints():
    h = Bk.lowpass_taps()
    n = np.arange(-4, 5)
    assert np.allclose(h, h[::-1], atol=0)
    assert abs(h.sum() - 1.0) < 1e-14                    # H(0) = 1
    assert abs(np.sum(h * n ** 2)) < 1e-14               # H''(0) = 0
    assert abs(np.sum(h * n ** 4)) < 1e-13               # H''''(0) = 0
    assert abs(np.sum(h * (-1.0) ** n)) < 1e-14          # H(pi) = 0
    assert abs(abs(_dtft(h, [np.pi / 2])[0]) - 1 / math.sqrt(2)) < 1e-14  # 3 dB
    w = np.linspace(-np.pi, np.pi, 41)
    np.testing.assert_allclose(Bk.H(w), _dtft(h, w).real, atol=1e-14)
    g = Bk.highpass_taps()
    np.testing.assert_allclose(g, ((-1.0) ** n) * h, atol=0)
    np.testing.assert_allclose(Bk.G(w), _dtft(g, w).real, atol=1e-14)


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_iterated_filters_match_convolutions(j):
    w = np.linspace(-np.pi, np.pi, 67)
    np.testing.assert_allclose(Bk.H_iter(j, w), _dtft(Bk.iterated_taps(j, False), w).real,
                               atol=1e-13)
    np.testing.assert_allclose(Bk.G_iter(j, w), _dtft(Bk.iterated_taps(j, True), w).real,
                               atol=1e-13)


def test_fan_filter():
    taps = Bk.fan_taps()
    assert taps.shape == (7, 7)
    w2, w1 = np.meshgrid(np.linspace(-np.pi, np.pi, 19), np.linspace(-np.pi, np.pi, 23),
                         indexing="ij")
    n2 = np.arange(7) - 3
    n1 = np.arange(7) - 3
    ref = np.zeros(w1.shape, dtype=complex)
    for a in range(7):
        for b in range(7):
            ref += taps[a, b] * np.exp(-1j * (w2 * n2[a] + w1 * n1[b]))
    np.testing.assert_allclose(Bk.fan(w1, w2), ref.real, atol=1e-14)
    assert np.abs(ref.imag).max() < 1e-14
    assert abs(Bk.fan(np.pi, 0.0) - 1.0) < 1e-15      # horizontal cone passes
    assert abs(Bk.fan(0.0, np.pi)) < 1e-15            # vertical cone stops
    d = np.linspace(-np.pi, np.pi, 13)
    np.testing.assert_allclose(Bk.fan(d, d), 0.5, atol=1e-15)   # cone boundary
    # half-band complementarity: P(w) + P(w + (pi, pi)) = 1
    np.testing.assert_allclose(Bk.fan(w1, w2) + Bk.fan(w1 + np.pi, w2 + np.pi), 1.0,
                               atol=1e-14)


@pytest.mark.parametrize("l,k", [(1, 0), (1, -2), (1, 1), (2, 3), (2, -4)])
def test_digital_shear_transfer_matches_literal_operator(l, k):
    N, M = 8, 8
    rng = np.random.default_rng(l * 10 + k)
    f = rng.standard_normal((N, M))
    lit = Bk.shear_spatial_literal(f, l, k)
    fast = np.fft.ifft(np.fft.fft(f, axis=1) * Bk.shear_transfer(l, k, N, M), axis=1)
    np.testing.assert_allclose(fast.real, lit, atol=1e-12)
    assert np.abs(fast.imag).max() < 1e-12


@pytest.mark.parametrize("levels,full,count", [
    ([1, 1], False, 17), ([1, 1, 2], False, 33), ([1, 1, 2, 2], False, 49),
    ([1, 1], True, 21), ([1], False, 9),
])
def test_filter_counts(levels, full, count):
    assert Bk.n_shearlets(levels, full) == count
    assert Bk.default_shear_levels(len(levels)) == levels or full or levels == [1]


def test_eq_3_2_count_with_default_levels():
    # Eq. 3.2, nShearlets = 2 sum_j (|K_j| - 1) + 1 with |K_j| = 2^{l_j+1} + 1
    for J, want in [(2, 17), (3, 33), (4, 49)]:
        lv = Bk.default_shear_levels(J)
        assert 2 * sum(2 ** (l + 1) for l in lv) + 1 == want
        b = Bk.shearlet_bank(32, 32, J)
        assert b["spectra"].shape == (want, 32, 32)


@pytest.fixture(scope="module")
def bank64():
    return Bk.shearlet_bank(64, 64, 3)


def test_bank_real_even_positive(bank64):
    S = bank64["spectra"]
    neg = np.roll(np.roll(S[:, ::-1, ::-1], 1, axis=1), 1, axis=2)
    np.testing.assert_array_equal(S, neg)            # exactly even
    W = bank64["dual_w"]
    assert W.min() > 1e-3 and np.isfinite(W).all()
    assert abs(S[0, 0, 0] - 1.0) < 1e-14            # low-pass carries DC
    assert np.abs(S[1:, 0, 0]).max() < 1e-14         # band-passes vanish at DC
    np.testing.assert_allclose(bank64["psi_hat"], T.tfftshift(S), atol=0)


def test_bank_cone_symmetry_and_index(bank64):
    S, idx = bank64["spectra"], bank64["idx"]
    assert tuple(idx[0]) == (0, 0, 0)
    pos = {tuple(r): i for i, r in enumerate(idx)}
    for (cone, j, k), i in pos.items():
        if cone == 2:
            np.testing.assert_allclose(S[i], S[pos[(1, j, k)]].T, atol=1e-13)
    # per scale: cone 1 k ascending then cone 2 k ascending
    for j in (1, 2, 3):
        ks1 = [r[2] for r in idx if r[0] == 1 and r[1] == j]
        ks2 = [r[2] for r in idx if r[0] == 2 and r[1] == j]
        l = Bk.default_shear_levels(3)[j - 1]
        assert ks1 == list(range(-2 ** l, 2 ** l + 1))
        assert ks2 == list(range(-2 ** l + 1, 2 ** l))


def test_bank_rms_is_spatial_norm(bank64):
    S = bank64["spectra"]
    spatial = np.fft.ifft2(S, axes=(-2, -1))
    assert np.abs(spatial.imag).max() < 1e-15
    np.testing.assert_allclose(bank64["rms"], np.sqrt(np.sum(spatial.real ** 2, axis=(1, 2))),
                               rtol=1e-12)


def test_bank_sheared_wedges_move_with_k(bank64):
    # The energy centroid slope w2/w1 of cone-1 filters increases with k.
    S, idx = bank64["spectra"], bank64["idx"]
    N = 64
    f = np.fft.fftfreq(N)
    w2, w1 = np.meshgrid(f, f, indexing="ij")
    sel = (w1 > 0)
    for j in (1, 2, 3):
        rows = [i for i, r in enumerate(idx) if r[0] == 1 and r[1] == j]
        slopes = []
        for i in rows:
            e = S[i] ** 2 * sel
            slopes.append(np.sum(e * w2 / np.maximum(w1, 1e-9)) / np.sum(e))
        assert np.all(np.diff(slopes) > 0), slopes


def test_rectangular_bank():
    b = Bk.shearlet_bank(32, 64, 2)
    S = b["spectra"]
    assert S.shape == (17, 32, 64)
    neg = np.roll(np.roll(S[:, ::-1, ::-1], 1, axis=1), 1, axis=2)
    np.testing.assert_array_equal(S, neg)
    assert b["dual_w"].min() > 1e-3


def test_white_noise_subband_std_is_sigma_rms():
    N, sigma = 128, 0.3
    b = Bk.shearlet_bank(N, N, 2)
    rng = np.random.default_rng(5)
    e = sigma * rng.standard_normal((4, N, N))
    c = np.fft.ifft2(np.fft.fft2(e)[:, None] * b["spectra"][None], axes=(-2, -1)).real
    std = c.std(axis=(0, 2, 3))
    np.testing.assert_allclose(std, sigma * b["rms"], rtol=0.03)
