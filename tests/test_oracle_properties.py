"""Property checks of the oracle over random sizes (CPU; hypothesis when
available): the paper's literal shifted form equals the natural-order form,
perfect reconstruction and adjointness hold for random Hermitian banks at
any size, and the discrete ray transform's adjoint is its transpose."""

import numpy as np
import pytest

from oracle import ray as OR
from oracle import transform as T

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


@hyp.settings(max_examples=40, deadline=None)
@hyp.given(N=st.integers(1, 13), M=st.integers(1, 13), K=st.integers(1, 4),
           seed=st.integers(0, 2 ** 31 - 1))
def test_shift_cancellation_and_frame_identities(N, M, K, seed):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((K, N, M))
    G = np.fft.fft2(g, axes=(-2, -1)) + 2.0            # Hermitian; the constant keeps W > 0
    psi_hat = np.conj(T.tfftshift(G))                  # the paper's centred layout
    f = rng.standard_normal((N, M))
    c_lit = T.decompose(f, psi_hat)
    c_nat = T.decompose_natural(f, G)
    scale = max(np.abs(c_nat).max(), 1e-300)
    assert np.abs(c_lit - c_nat).max() <= 1e-11 * scale
    assert np.abs(c_nat.imag).max() <= 1e-11 * scale
    rec = T.reconstruct_natural(c_nat.real, G)
    assert np.abs(rec - f).max() <= 1e-10 * max(np.abs(f).max(), 1.0)
    cc = rng.standard_normal((K, N, M))
    lhs = np.sum(c_nat.real * cc)
    rhs = np.sum(f * T.reconstruct_natural(cc, G, weights=False).real)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)


@hyp.settings(max_examples=25, deadline=None)
@hyp.given(N=st.integers(2, 24), A=st.integers(1, 12), D=st.integers(1, 40),
           seed=st.integers(0, 2 ** 31 - 1))
def test_ray_adjoint_identity(N, A, D, seed):
    rng = np.random.default_rng(seed)
    x, y = rng.standard_normal((N, N)), rng.standard_normal((A, D))
    lhs = np.sum(OR.forward(x, A, D) * y)
    rhs = np.sum(x * OR.adjoint(y, N))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@hyp.settings(max_examples=15, deadline=None)
@hyp.given(N=st.integers(4, 20), q=st.integers(1, 6), seed=st.integers(0, 2 ** 31 - 1))
def test_ray_quarter_turn(N, q, seed):
    # A = 4q angles: phi + pi/2 is again a grid angle
    A = 4 * q
    D = int(np.ceil(np.sqrt(2) * N))
    f = np.random.default_rng(seed).standard_normal((N, N))
    pf, pg = OR.forward(f, A, D), OR.forward(np.rot90(f, -1).copy(), A, D)
    h = A // 2
    for a in range(A):
        want = pf[a - h] if a >= h else pf[a + h][::-1]
        assert np.abs(pg[a] - want).max() <= 1e-11 * max(np.abs(pf).max(), 1.0)
