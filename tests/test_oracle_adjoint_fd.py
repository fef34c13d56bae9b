"""Finite differences (float64, eps = 1e-3) pin the oracle's adjoints, which
the GPU backward passes are then compared against (CPU only)."""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as T


@pytest.mark.parametrize("n", [16, 32])
def test_fd_gradient_of_decomposition_is_adjoint(n):
    b = Bk.shearlet_bank(n, n, 2)
    psi = b["psi_hat"]
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n))
    w = rng.standard_normal((len(psi), n, n))
    L = lambda z: float(np.sum(w * T.decompose(z, psi).real))
    g = T.adjoint(w, psi).real
    eps = 1e-3
    for _ in range(5):
        v = rng.standard_normal((n, n))
        fd = (L(x + eps * v) - L(x - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) <= 1e-9 * max(1.0, abs(fd))


@pytest.mark.parametrize("n", [16, 32])
def test_fd_gradient_of_reconstruction_is_dual_decomposition(n):
    b = Bk.shearlet_bank(n, n, 2)
    psi = b["psi_hat"]
    rng = np.random.default_rng(n + 1)
    c = rng.standard_normal((len(psi), n, n))
    w = rng.standard_normal((n, n))
    L = lambda z: float(np.sum(w * T.reconstruct(z, psi).real))
    g = T.decompose_dual(w, psi).real
    eps = 1e-3
    for _ in range(5):
        v = rng.standard_normal(c.shape)
        fd = (L(c + eps * v) - L(c - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) <= 1e-9 * max(1.0, abs(fd))
