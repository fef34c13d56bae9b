"""FP64 oracle: the digital shearlet filter bank (Sec. 2.1 and 3.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper builds its default system from two third-party filters (a MATLAB
``maxflat`` design and the contourlet toolbox's ``dmaxflat4`` fan filter)
whose coefficients it does not print.  This module designs both from their
published definitions instead, then follows the paper's construction:

* 1D low-pass h (Sec. 3.4: order 8, i.e. 9 symmetric taps, maximally flat,
  3 dB point at half the Nyquist frequency).  Cosine form
  ``H(w) = b0 + sum_{m=1..4} b_m cos(m w)``; the five coefficients solve
  H(0)=1, H''(0)=0, H''''(0)=0 (flat at DC), H(pi)=0, H(pi/2)=1/sqrt(2).
* high-pass g(n) = (-1)^n h(n), the mirror filter (Sec. 3.4).
* iterated filters (Sec. 2.1): ``h_j(w) = prod_{k<j} h(2^k w)``,
  ``g_j(w) = g(2^{j-1} w) h_{j-1}(w)``, ``h_0 = 1``.
* fan filter P (Sec. 3.4, after da Cunha-Zhou-Do): the McClellan transform of
  the 1D maximally flat half-band polynomial
  ``Hmf(t) = ((1+t)/2)^2 (2 - t)`` with ``t = (cos w2 - cos w1)/2``.  With
  ``cos w1 + cos w2`` this is a diamond filter; the modulation (-1)^{n1} of
  the paper's ``modulate2`` turns it into the fan that passes |w2| < |w1|.
* unsheared shearlet of scale j (Eq. 2.6 before shearing, ``p_j * W_j``):
  ``P(a1 w1, a2 w2) g_{J-j}(w1) h_{J-j-1+l_j}(w2)`` with
  ``a1 = 2^{J-j-1}`` and ``a2 = a1 2^{l_j}`` (``l_j`` = shear level of scale
  j).  The fan dilation makes the wedge slope 2^{-l_j}.
* digital shear (Eqs. 2.4-2.5): along x1, upsample by 2^l, convolve with
  2^l h_l, shift row x2 by k x2 fine samples, convolve with h_l, downsample
  by 2^l.  On the circular N x M grid this equals multiplying the row
  spectrum by ``sum_r h_l(w_r)^2 exp(+i w_r k x2)`` over the 2^l aliases
  ``w_r = 2 pi (p1 + r M) / (M 2^l)`` of column frequency p1.
* cone 2 is cone 1 built on the transposed grid and transposed back; the
  low-pass is ``h_J (x) h_J``.

Readings (where the paper is garbled or silent):

* shear level of scale j (0-based, coarse to fine) defaults to
  ``ceil((j+1)/2)``; shears ``k = -2^l..2^l`` in cone 1 and, unless
  ``full``, ``k = -2^l+1..2^l-1`` in cone 2, giving 17 / 33 / 49 filters for
  2 / 3 / 4 scales.
* filter order: 0 = low-pass; then for each scale coarse to fine, cone 1 with
  k ascending, then cone 2 with k ascending.  ``idx[i] = (cone, scale, k)``
  with scale counted from 1 and the low-pass (0, 0, 0).
* every spectrum is real and even (point-symmetric real filter): the built
  spectrum's real part is kept and even-symmetrised, which is exactly the
  point-symmetrisation of the spatial filter.

Spectra are returned in natural DFT order (index 0 = zero frequency) with
shape [K, N, M], and centred (``fftshift``) for the paper's layout.
"""

from __future__ import annotations

import math
from itertools import product

import numpy as np


# ------------------------------------------------------------- 1D filters
def lowpass_cosine_coeffs() -> np.ndarray:
    """b0..b4 of the 9-tap maximally flat low-pass (module docstring)."""
    m = np.arange(5, dtype=np.float64)
    A = np.stack([
        np.ones(5),                 # H(0) = 1
        m ** 2,                     # H''(0) = 0   (d^2/dw^2 cos(mw) = -m^2)
        m ** 4,                     # H''''(0) = 0
        (-1.0) ** m,                # H(pi) = 0
        np.cos(m * np.pi / 2),      # H(pi/2) = 1/sqrt(2)
    ])
    rhs = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / math.sqrt(2.0)])
    return np.linalg.solve(A, rhs)


def lowpass_taps() -> np.ndarray:
    """h(n), n = -4..4 (index 4 is n = 0)."""
    b = lowpass_cosine_coeffs()
    h = np.zeros(9)
    h[4] = b[0]
    for k in range(1, 5):
        h[4 + k] = h[4 - k] = b[k] / 2.0
    return h


def highpass_taps() -> np.ndarray:
    """g(n) = (-1)^n h(n), n = -4..4."""
    n = np.arange(-4, 5)
    return ((-1.0) ** n) * lowpass_taps()


def H(w) -> np.ndarray:
    """Frequency response of h (real, 2 pi periodic)."""
    b = lowpass_cosine_coeffs()
    w = np.asarray(w, dtype=np.float64)
    return b[0] + sum(b[k] * np.cos(k * w) for k in range(1, 5))


def G(w) -> np.ndarray:
    """Frequency response of g: H(w + pi)."""
    return H(np.asarray(w, dtype=np.float64) + np.pi)


def H_iter(j: int, w) -> np.ndarray:
    """h_j(w) = prod_{k=0}^{j-1} H(2^k w), h_0 = 1."""
    w = np.asarray(w, dtype=np.float64)
    out = np.ones_like(w)
    for k in range(j):
        out = out * H((2.0 ** k) * w)
    return out


def G_iter(j: int, w) -> np.ndarray:
    """g_j(w) = G(2^{j-1} w) h_{j-1}(w), j >= 1."""
    w = np.asarray(w, dtype=np.float64)
    return G((2.0 ** (j - 1)) * w) * H_iter(j - 1, w)


def iterated_taps(j: int, high: bool) -> np.ndarray:
    """Spatial taps of h_j (or g_j) by explicit convolutions, centred.

    h_j = h * (h up 2) * ... * (h up 2^{j-1}); g_j = (g up 2^{j-1}) * h_{j-1}.
    Used by tests to pin :func:`H_iter` / :func:`G_iter`.
    """
    def up(t, f):
        out = np.zeros((len(t) - 1) * f + 1)
        out[::f] = t
        return out
    h = lowpass_taps()
    acc = np.array([1.0])
    for k in range(j - 1 if high else j):
        acc = np.convolve(acc, up(h, 2 ** k))
    if high:
        acc = np.convolve(acc, up(highpass_taps(), 2 ** (j - 1)))
    return acc


# ------------------------------------------------------------- fan filter
def maxflat_halfband(t) -> np.ndarray:
    """((1+t)/2)^2 (2 - t): maximally flat at t=1 and t=-1, Hmf(t)+Hmf(-t)=1."""
    t = np.asarray(t, dtype=np.float64)
    return ((1.0 + t) / 2.0) ** 2 * (2.0 - t)


def fan(w1, w2) -> np.ndarray:
    """Fan filter P(w1, w2): passes |w2| < |w1| (x1 = horizontal axis)."""
    t = (np.cos(w2) - np.cos(w1)) / 2.0
    return maxflat_halfband(t)


def fan_taps() -> np.ndarray:
    """Spatial 7x7 taps of P, [n2, n1] centred at (3, 3), built by 2D
    polynomial convolution of the McClellan kernel (pins :func:`fan`)."""
    # t <-> kernel: 1/4 at (0, +-1) [cos w2 term uses n2] ... written as arrays
    T = np.zeros((3, 3))
    T[0, 1] = T[2, 1] = 0.25      # + cos(w2)/2  (n2 = +-1)
    T[1, 0] = T[1, 2] = -0.25     # - cos(w1)/2  (n1 = +-1)
    one = np.zeros((3, 3))
    one[1, 1] = 1.0

    def conv2(a, b):
        out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
        for (i, j) in product(range(b.shape[0]), range(b.shape[1])):
            out[i:i + a.shape[0], j:j + a.shape[1]] += b[i, j] * a
        return out
    a = (one + T) / 2.0                   # (1+t)/2
    b = 2.0 * one - T                     # 2 - t
    return conv2(conv2(a, a), b)


# ----------------------------------------------------------- shear levels
def default_shear_levels(n_scales: int) -> list[int]:
    return [int(math.ceil((j + 1) / 2)) for j in range(n_scales)]


def n_shearlets(shear_levels, full: bool = False) -> int:
    """1 + sum_j (cone 1: 2^{l+1}+1 shears, cone 2: 2^{l+1}-1 or +1)."""
    k = 1
    for l in shear_levels:
        k += (2 ** (l + 1) + 1) + (2 ** (l + 1) + (1 if full else -1))
    return k


# ---------------------------------------------------------- digital shear
def shear_transfer(l: int, k: int, N: int, M: int) -> np.ndarray:
    """[N, M] multiplier on (x2 row, p1 column frequency) of S^d_k at level l."""
    U = 2 ** l
    c2 = np.arange(N)
    c2 = np.where(c2 < N // 2, c2, c2 - N).astype(np.float64)[:, None]
    out = np.zeros((N, M), dtype=np.complex128)
    p1 = np.arange(M, dtype=np.float64)[None, :]
    for r in range(U):
        w = 2.0 * np.pi * (p1 + r * M) / (M * U)
        out += (H_iter(l, w) ** 2) * np.exp(1j * w * k * c2)
    return out


def shear_spatial_literal(f: np.ndarray, l: int, k: int) -> np.ndarray:
    """Eqs. 2.4-2.5 on the circular grid by explicit loops (tiny inputs).

    Upsample along x1 (axis 1) by 2^l, circularly convolve with 2^l h_l,
    shift row x2 by k*x2 fine samples (g[q] = f[q + k x2]), convolve with
    h_l, downsample by 2^l.  Pins :func:`shear_transfer`.
    """
    N, M = f.shape
    U = 2 ** l
    L = M * U
    hl = iterated_taps(l, high=False)
    half = (len(hl) - 1) // 2

    def cconv_row(row, taps, gain):
        out = np.zeros(L)
        for q in range(L):
            s = 0.0
            for t in range(len(taps)):
                s += taps[t] * row[(q - (t - half)) % L]
            out[q] = gain * s
        return out
    res = np.zeros((N, M))
    for x2 in range(N):
        c2 = x2 if x2 < N // 2 else x2 - N
        up = np.zeros(L)
        up[::U] = f[x2]
        a = cconv_row(up, hl, float(U))
        b = np.array([a[(q + k * c2) % L] for q in range(L)])
        c = cconv_row(b, hl, 1.0)
        res[x2] = c[::U]
    return res


# ------------------------------------------------------------------ bank
def _grid(N: int, M: int):
    w2 = (2.0 * np.pi * np.arange(N) / N)[:, None]
    w1 = (2.0 * np.pi * np.arange(M) / M)[None, :]
    return w2, w1


def unsheared(j: int, J: int, l: int, N: int, M: int) -> np.ndarray:
    """psi_hat_{j,0} = P(a1 w1, a2 w2) g_{J-j}(w1) h_{J-j-1+l}(w2), natural."""
    w2, w1 = _grid(N, M)
    a1 = 2.0 ** (J - j - 1)
    a2 = a1 * 2.0 ** l
    return fan(a1 * w1, a2 * w2) * G_iter(J - j, w1) * H_iter(J - j - 1 + l, w2)


def _cone1(j, J, l, k, N, M):
    base = unsheared(j, J, l, N, M)
    mixed = np.fft.ifft(base, axis=0)               # x2 rows, p1 columns
    Gk = np.fft.fft(mixed * shear_transfer(l, k, N, M), axis=0)
    return _real_even(Gk)


def _real_even(Gc: np.ndarray) -> np.ndarray:
    Gr = Gc.real
    neg = np.roll(np.roll(Gr[::-1, ::-1], 1, axis=0), 1, axis=1)   # G(-p)
    return 0.5 * (Gr + neg)


def shearlet_bank(rows: int, cols: int, n_scales: int, shear_levels=None,
                  full: bool = False) -> dict:
    """The digital shearlet system (``getshearletsystem2D`` of Sec. 3.4).

    Returns dict with
      ``spectra``  [K, rows, cols] float64, natural DFT order, real and even;
      ``psi_hat``  the same, centred (the paper's layout);
      ``idx``      [K, 3] int (cone, scale, shear);
      ``rms``      [K] = ||psi_i||_2 = sqrt(sum G_i^2 / (rows cols));
      ``dual_w``   [rows, cols] natural order, W = sum_i G_i^2.
    """
    N, M = rows, cols
    J = n_scales
    if shear_levels is None:
        shear_levels = default_shear_levels(J)
    shear_levels = list(shear_levels)
    w2, w1 = _grid(N, M)
    spectra = [H_iter(J, w1) * H_iter(J, w2)]
    idx = [(0, 0, 0)]
    for j in range(J):
        l = shear_levels[j]
        for k in range(-2 ** l, 2 ** l + 1):
            spectra.append(_cone1(j, J, l, k, N, M))
            idx.append((1, j + 1, k))
        kmax = 2 ** l if full else 2 ** l - 1
        for k in range(-kmax, kmax + 1):
            spectra.append(_cone1(j, J, l, k, M, N).T.copy())
            idx.append((2, j + 1, k))
    S = np.stack(spectra).astype(np.float64)
    S[0] = _real_even(S[0].astype(np.complex128))
    W = np.sum(S ** 2, axis=0)
    rms = np.sqrt(np.sum(S ** 2, axis=(1, 2)) / (N * M))
    return {
        "spectra": S,
        "psi_hat": np.fft.fftshift(S, axes=(-2, -1)),
        "idx": np.asarray(idx, dtype=np.int32),
        "rms": rms,
        "dual_w": W,
    }
