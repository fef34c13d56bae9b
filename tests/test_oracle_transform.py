"""Pins for the FP64 oracle's transform (CPU only).

Each check compares the oracle against something other than itself: the
shift lists printed in Sec. 3.3, the DFT's defining double sum, a direct
spatial correlation (Def. 2.6), closed-form identities (perfect
reconstruction, adjointness, Parseval) and special banks whose answer is
known.  ``test_planted_mistakes_are_caught`` plants plausible mistakes in a
copy of the oracle and checks that these pins catch every one of them.
"""

import numpy as np
import pytest

from oracle import transform as T

RNG = np.random.default_rng(12345)


def _rand_complex(shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _inner(a, b):
    return np.vdot(b.ravel(), a.ravel())  # sum a * conj(b)


def _random_bank(K, N, M, rng=RNG):
    """Random complex filters with full support, as centred spatial arrays."""
    psi_centre = _rand_complex((K, N, M), rng)
    psi_paper = T.tfftshift(psi_centre)          # centre moved to n//2
    psi_hat = np.stack([T.fourier(p) for p in psi_paper])
    return psi_centre, psi_hat


# ------------------------------------------------------------- Sec. 3.3
def test_shift_lists_golden_file():
    """tests/golden/shift_indices.txt: the gather lists of Sec. 3.3's shift
    definitions written out by hand for n = 1..8."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "shift_indices.txt")
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for line in rows:
        n, fwd, inv = (part.split() for part in line.split("|"))
        n = int(n[0])
        assert list(T.tfftshift_indices(n)) == [int(v) for v in fwd]
        assert list(T.itfftshift_indices(n)) == [int(v) for v in inv]
        a = np.arange(n)
        assert list(np.fft.fftshift(a)) == [int(v) for v in fwd]     # the library routine agrees
        assert list(np.fft.ifftshift(a)) == [int(v) for v in inv]


def test_shift_lists_printed_example():
    # Sec. 3.3: p2 = (n+1)//2 for tfftshift, n - (n+1)//2 for itfftshift.
    assert list(T.tfftshift_indices(5)) == [3, 4, 0, 1, 2]
    assert list(T.itfftshift_indices(5)) == [2, 3, 4, 0, 1]
    assert list(T.tfftshift_indices(4)) == [2, 3, 0, 1]


@pytest.mark.parametrize("n", range(1, 13))
def test_shifts_match_library_fftshift(n):
    a = np.arange(n * 3).reshape(3, n) * 1.0
    np.testing.assert_array_equal(T.tfftshift(a, axes=(1,)), np.fft.fftshift(a, axes=1))
    np.testing.assert_array_equal(T.itfftshift(a, axes=(1,)), np.fft.ifftshift(a, axes=1))
    np.testing.assert_array_equal(T.itfftshift(T.tfftshift(a)), a)


@pytest.mark.parametrize("shape", [(8, 8), (6, 4), (5, 7)])
def test_fft2_primitive_matches_definition(shape):
    f = _rand_complex(shape)
    np.testing.assert_allclose(np.fft.fft2(f), T.dft2_direct(f), rtol=0, atol=1e-11)


# ------------------------------------------------------------ Def. 2.6
@pytest.mark.parametrize("shape", [(16, 16), (8, 12), (9, 7)])
def test_decompose_is_spatial_correlation(shape):
    N, M = shape
    psi_c, psi_hat = _random_bank(3, N, M)
    f = RNG.standard_normal((N, M))
    c = T.decompose(f, psi_hat)
    for i in range(3):
        ref = T.correlate_direct(f, psi_c[i])
        np.testing.assert_allclose(c[i], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_delta_bank_gives_circular_shifts():
    N, M = 12, 10
    f = RNG.standard_normal((N, M))
    shifts = [(0, 0), (3, -2), (-5, 4)]
    psi_c = np.zeros((3, N, M))
    for i, (a, b) in enumerate(shifts):
        psi_c[i, a % N, b % M] = 1.0
    psi_hat = np.stack([T.fourier(T.tfftshift(p)) for p in psi_c])
    c = T.decompose(f, psi_hat)
    for i, (a, b) in enumerate(shifts):
        # c(m) = f(m + s)
        want = np.roll(np.roll(f, -a, axis=0), -b, axis=1)
        np.testing.assert_allclose(c[i].real, want, atol=1e-13)
        assert np.abs(c[i].imag).max() < 1e-13


def test_identity_bank():
    N, M = 16, 8
    f = RNG.standard_normal((N, M))
    psi_hat = np.ones((1, N, M))
    np.testing.assert_allclose(T.decompose(f, psi_hat)[0], f, atol=1e-14)
    c = RNG.standard_normal((1, N, M))
    np.testing.assert_allclose(T.reconstruct(c, psi_hat), c[0], atol=1e-14)


# ------------------------------------------------- closed-form identities
@pytest.mark.parametrize("shape", [(16, 16), (8, 12), (9, 7)])
def test_perfect_reconstruction(shape):
    N, M = shape
    _, psi_hat = _random_bank(5, N, M)
    f = RNG.standard_normal((N, M))
    rec = T.reconstruct(T.decompose(f, psi_hat), psi_hat)
    np.testing.assert_allclose(rec, f, rtol=0, atol=1e-12 * np.abs(f).max())


@pytest.mark.parametrize("shape", [(16, 16), (9, 7)])
def test_adjoint_identities(shape):
    N, M = shape
    _, psi_hat = _random_bank(4, N, M)
    f = _rand_complex((N, M))
    c = _rand_complex((4, N, M))
    lhs = _inner(T.decompose(f, psi_hat), c)
    rhs = _inner(f, T.adjoint(c, psi_hat))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = _inner(T.reconstruct(c, psi_hat), f)
    rhs = _inner(c, T.decompose_dual(f, psi_hat))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_frame_identity_parseval():
    N, M = 16, 12
    _, psi_hat = _random_bank(4, N, M)
    f = RNG.standard_normal((N, M))
    c = T.decompose(f, psi_hat)
    lhs = np.sum(np.abs(c) ** 2)
    rhs = np.sum(T.dual_frame_weights(psi_hat) * np.abs(T.fourier(f)) ** 2) / (N * M)
    assert abs(lhs - rhs) <= 1e-12 * lhs


# ------------------------------------------------------- natural order
@pytest.mark.parametrize("shape", [(16, 16), (8, 12)])
def test_natural_order_form_equals_literal(shape):
    N, M = shape
    _, psi_hat = _random_bank(3, N, M)
    f = RNG.standard_normal((N, M))
    G = T.centred_to_natural(psi_hat)
    np.testing.assert_allclose(T.decompose_natural(f, G), T.decompose(f, psi_hat),
                               atol=1e-12)
    c = _rand_complex((3, N, M))
    np.testing.assert_allclose(T.reconstruct_natural(c, G), T.reconstruct(c, psi_hat),
                               atol=1e-12)
    np.testing.assert_allclose(T.reconstruct_natural(c, G, weights=False),
                               T.adjoint(c, psi_hat), atol=1e-12)


def test_real_even_bank_gives_real_coefficients():
    N = 16
    rng = np.random.default_rng(7)
    g = rng.standard_normal((3, N, N))
    # point-symmetric real spatial filters -> real even spectra
    g = 0.5 * (g + np.roll(np.roll(g[:, ::-1, ::-1], 1, axis=1), 1, axis=2))
    G = np.fft.fft2(g).real
    psi_hat = np.fft.fftshift(G, axes=(-2, -1))
    f = rng.standard_normal((N, N))
    c = T.decompose(f, psi_hat)
    assert np.abs(c.imag).max() < 1e-13 * np.abs(c.real).max()


# ------------------------------------------------------ planted mistakes
def _pins(mod):
    """Run the pins above against module-like ``mod``; return failures."""
    fails = []
    rng = np.random.default_rng(99)
    for (N, M) in [(8, 8), (7, 5)]:
        psi_c = _rand_complex((3, N, M), rng)
        psi_hat = np.stack([T.fourier(p) for p in T.tfftshift(psi_c)])
        f = rng.standard_normal((N, M))
        c = mod.decompose(f, psi_hat)
        if any(np.abs(c[i] - T.correlate_direct(f, psi_c[i])).max() > 1e-9 for i in range(3)):
            fails.append("correlation")
        if np.abs(mod.reconstruct(mod.decompose(f, psi_hat), psi_hat) - f).max() > 1e-9:
            fails.append("pr")
        fc = _rand_complex((N, M), rng)
        cc = _rand_complex((3, N, M), rng)
        a, b = _inner(mod.decompose(fc, psi_hat), cc), _inner(fc, mod.adjoint(cc, psi_hat))
        if abs(a - b) > 1e-9 * abs(a):
            fails.append("adjoint")
        a, b = _inner(mod.reconstruct(cc, psi_hat), fc), _inner(cc, mod.decompose_dual(fc, psi_hat))
        if abs(a - b) > 1e-9 * abs(a):
            fails.append("adjoint-dual")
    return fails


class _Mutant:
    def __init__(self, **over):
        self.decompose = T.decompose
        self.reconstruct = T.reconstruct
        self.adjoint = T.adjoint
        self.decompose_dual = T.decompose_dual
        self.__dict__.update(over)


def _dec_conj_on_image(f, psi_hat):          # the algorithm box's placement
    X = T.fourier(f)
    return np.stack([T.inverse_fourier(psi_hat[i] * np.conj(X)) for i in range(len(psi_hat))])


def _dec_swapped_shifts(f, psi_hat):
    X = T.itfftshift(np.fft.fft2(T.tfftshift(f)))
    return np.stack([T.itfftshift(np.fft.ifft2(T.tfftshift(X * np.conj(p)))) for p in psi_hat])


def _rec_no_weights(c, psi_hat):
    return T.adjoint(c, psi_hat)


def _adj_conj_filter(c, psi_hat):
    acc = sum(T.fourier(c[i]) * np.conj(psi_hat[i]) for i in range(len(psi_hat)))
    return T.inverse_fourier(acc)


def _dual_no_weights(y, psi_hat):
    return T.decompose(y, psi_hat)


def _dec_dropped_filter(f, psi_hat):
    out = T.decompose(f, psi_hat)
    out[-1] = 0
    return out


@pytest.mark.parametrize("mutant", [
    _Mutant(decompose=_dec_conj_on_image),
    _Mutant(decompose=_dec_swapped_shifts),
    _Mutant(reconstruct=_rec_no_weights),
    _Mutant(adjoint=_adj_conj_filter),
    _Mutant(decompose_dual=_dual_no_weights),
    _Mutant(decompose=_dec_dropped_filter),
])
def test_planted_mistakes_are_caught(mutant):
    assert _pins(mutant), "a planted mistake passed every pin"


def test_unmutated_oracle_passes_pins():
    assert _pins(_Mutant()) == []
