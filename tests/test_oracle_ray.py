"""Pins for the FP64 ray-transform oracle of Sec. 4.4 (CPU only).

The discrete transform is a reading (Joseph's method on [-1, 1]^2, see
``oracle/ray.py``).  It is checked against what the continuous definition
fixes: the exact line integrals of ellipses (first-order convergence as the
grid is refined), the integral of an image that is constant along y (a
textbook linear interpolation), and the rotation identity R(f o rot)(s, phi)
= R f(s, phi - pi/2), which ties the row-sampled and the column-sampled
angles to each other.
"""

import numpy as np
import pytest

from oracle import ray as R
from paper_2006_04591_gb300 import synth

ELL = np.array([[1.0, 0.5, 0.25, 0.2, -0.3, 0.4], [0.5, 0.2, 0.1, -0.4, 0.35, 1.1]])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_converges_to_exact_ellipse_integrals():
    errs = []
    for N in (64, 128, 256):
        A, D = 30, int(np.ceil(np.sqrt(2) * N))
        p = R.forward(R.ellipse_image(ELL, N, 8), A, D)
        errs.append(_rel(p, R.ellipse_sinogram(ELL, A, D)))
    assert errs[-1] < 0.012
    # first order in h: each halving of the pixel size about halves the error
    assert 1.6 < errs[0] / errs[1] < 2.5 and 1.6 < errs[1] / errs[2] < 2.5


def test_shepp_logan_sinogram():
    N, A, D = 256, 30, 363
    tab = synth.shepp_logan()
    p = R.forward(R.ellipse_image(tab, N, 8), A, D)
    assert _rel(p, R.ellipse_sinogram(tab, A, D)) < 0.02


def test_image_constant_along_y_integrates_to_twice_the_profile():
    # at phi = 0 the rays are the vertical lines x = s: the integral over
    # y in [-1, 1] of f(x) is 2 f(x), f linear between pixel centres and
    # falling to 0 half a pixel outside the image
    N, A, D = 32, 6, 50
    g = R.geometry(N, A, D)
    prof = np.random.default_rng(4).uniform(0, 1, N)
    f = np.tile(prof, (N, 1))
    xs = np.concatenate([[g["x"][0] - g["h"]], g["x"], [g["x"][-1] + g["h"]]])
    want = 2.0 * np.interp(g["s"], xs, np.concatenate([[0.0], prof, [0.0]]))
    np.testing.assert_allclose(R.forward(f, A, D)[0], want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,A", [(32, 30), (48, 12)])
def test_quarter_turn_maps_row_sampling_to_column_sampling(N, A):
    D = int(np.ceil(np.sqrt(2) * N))
    f = np.random.default_rng(5).standard_normal((N, N))
    g = np.rot90(f, -1)                       # g(x, y) = f(y, -x)
    pf, pg = R.forward(f, A, D), R.forward(g.copy(), A, D)
    q = A // 2                                # phi + pi/2 = phi_{a + q}
    for a in range(A):
        want = pf[a - q] if a >= q else pf[a + q][::-1]   # R(s, phi - pi) = R(-s, phi)
        np.testing.assert_allclose(pg[a], want, rtol=0, atol=1e-12 * np.abs(pf).max())


def test_adjoint_is_transpose():
    N, A, D = 40, 17, 57
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal((3, N, N)), rng.standard_normal((3, A, D))
    lhs = np.sum(R.forward(x, A, D) * y)
    rhs = np.sum(x * R.adjoint(y, N))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
