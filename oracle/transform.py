"""FP64 oracle: the shearlet decomposition, reconstruction and adjoint.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (all from the paper):

* Sec. 3.3: the digital Fourier transform of an image is
  ``Fourier(f) = fftshift(fft2(ifftshift(f)))`` and its inverse
  ``InverseFourier(F) = fftshift(ifft2(ifftshift(F)))``.  The two shifts are
  the index permutations printed in Sec. 3.3: ``tfftshift`` rolls by
  ``p2 = (n+1)//2`` and ``itfftshift`` by ``p2 = n - (n+1)//2`` along each of
  the two image axes.
* Sec. 3.4, decomposition listing: coefficient i is
  ``InverseFourier(Fourier(f) * conj(psi_hat_i))``.  (The algorithm box puts
  the conjugate on the image spectrum instead; the listing's form is the one
  for which reconstruction inverts decomposition, so it is the one used.)
* Sec. 3.4, reconstruction listing: ``InverseFourier((sum_i
  Fourier(c_i) * psi_hat_i) / W)`` with the dual frame weights
  ``W = sum_i |psi_hat_i|^2`` (Eq. 2.7 written in the Fourier domain).
* The adjoint of the decomposition is the reconstruction without ``/ W``; the
  adjoint of the reconstruction ("dual-weighted decomposition") is the
  decomposition with ``conj(psi_hat_i) / W``.

Filter spectra ``psi_hat`` are centred (zero frequency at index n//2 after
``fftshift``), shape ``[K, N, M]``, complex or real, exactly the paper's
``[1, N, M, nShearlets]`` tensor with the channel axis moved first.
Coefficients have shape ``[K, N, M]``; the paper's ``coeffs[0, y, x, i]`` is
``c[i, y, x]`` here.

The natural-order functions drop both shifts.  The frequency-side pair
(``tfftshift`` of the image spectrum, ``itfftshift`` of the product) is a
permutation applied to both factors and undone, so it moves onto the filter:
``G_i = itfftshift(conj(psi_hat_i))``.  The space-side pair is a circular
translation of the image by ``p2`` before the filtering and back after it,
and circular filtering commutes with translations.  Hence
``c_i = ifft2(fft2(f) * G_i)`` at every size, odd or even (for even sizes it
is also the cancellation of the two ``(-1)^(k1+k2)`` modulations).  These
functions exist so that a test can check that algebra, and so that banks
given in natural order (the CUDA library's layout) can be fed to the oracle.
"""

from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- Sec. 3.3
def tfftshift_indices(n: int) -> np.ndarray:
    """Gather list of ``tfftshift`` along an axis of length n (Sec. 3.3)."""
    p2 = (n + 1) // 2
    return np.concatenate((np.arange(p2, n), np.arange(p2)))


def itfftshift_indices(n: int) -> np.ndarray:
    """Gather list of ``itfftshift`` along an axis of length n (Sec. 3.3)."""
    p2 = n - (n + 1) // 2
    return np.concatenate((np.arange(p2, n), np.arange(p2)))


def tfftshift(a: np.ndarray, axes=(-2, -1)) -> np.ndarray:
    """Forward Fourier shift by gathering along each axis (Sec. 3.3)."""
    for ax in axes:
        a = np.take(a, tfftshift_indices(a.shape[ax]), axis=ax)
    return a


def itfftshift(a: np.ndarray, axes=(-2, -1)) -> np.ndarray:
    """Inverse Fourier shift by gathering along each axis (Sec. 3.3)."""
    for ax in axes:
        a = np.take(a, itfftshift_indices(a.shape[ax]), axis=ax)
    return a


def fourier(f: np.ndarray) -> np.ndarray:
    """Centred 2D DFT over the last two axes: fftshift(fft2(ifftshift f))."""
    return tfftshift(np.fft.fft2(itfftshift(np.asarray(f, dtype=np.complex128)),
                                 axes=(-2, -1)))


def inverse_fourier(F: np.ndarray) -> np.ndarray:
    """Centred inverse 2D DFT: fftshift(ifft2(ifftshift F))."""
    return tfftshift(np.fft.ifft2(itfftshift(np.asarray(F, dtype=np.complex128)),
                                  axes=(-2, -1)))


# ---------------------------------------------------------------- Sec. 3.4
def dual_frame_weights(psi_hat: np.ndarray) -> np.ndarray:
    """W = sum_i |psi_hat_i|^2 (the ``tfdualFrameWeights`` of Sec. 3.4)."""
    return np.sum(np.abs(np.asarray(psi_hat)) ** 2, axis=0)


def decompose(f: np.ndarray, psi_hat: np.ndarray) -> np.ndarray:
    """Shearlet decomposition of one image (Sec. 3.4, decomposition listing).

    f: [N, M] real or complex.  psi_hat: [K, N, M] centred spectra.
    Returns complex128 [K, N, M].
    """
    X = fourier(f)
    K = psi_hat.shape[0]
    out = np.empty((K,) + X.shape, dtype=np.complex128)
    for i in range(K):
        out[i] = inverse_fourier(X * np.conj(psi_hat[i]))
    return out


def reconstruct(c: np.ndarray, psi_hat: np.ndarray) -> np.ndarray:
    """Shearlet reconstruction (Sec. 3.4, reconstruction listing).

    c: [K, N, M].  Returns complex128 [N, M].
    """
    K = psi_hat.shape[0]
    acc = np.zeros(psi_hat.shape[1:], dtype=np.complex128)
    for i in range(K):
        acc += fourier(c[i]) * psi_hat[i]
    return inverse_fourier(acc / dual_frame_weights(psi_hat))


def adjoint(c: np.ndarray, psi_hat: np.ndarray) -> np.ndarray:
    """Adjoint of :func:`decompose`: the reconstruction without 1/W."""
    K = psi_hat.shape[0]
    acc = np.zeros(psi_hat.shape[1:], dtype=np.complex128)
    for i in range(K):
        acc += fourier(c[i]) * psi_hat[i]
    return inverse_fourier(acc)


def decompose_dual(y: np.ndarray, psi_hat: np.ndarray) -> np.ndarray:
    """Adjoint of :func:`reconstruct`: decomposition with conj(psi_hat_i)/W."""
    X = fourier(y) / dual_frame_weights(psi_hat)
    K = psi_hat.shape[0]
    out = np.empty((K,) + X.shape, dtype=np.complex128)
    for i in range(K):
        out[i] = inverse_fourier(X * np.conj(psi_hat[i]))
    return out


# ------------------------------------------------------------ batched, real
def decompose_batch(x: np.ndarray, psi_hat: np.ndarray, dual: bool = False):
    """[B, N, M] real -> ([B, K, N, M] real part, max |imag| over all).

    For real images and real, even spectra the imaginary part is zero up to
    rounding; it is returned as a diagnostic.
    """
    fn = decompose_dual if dual else decompose
    outs = [fn(xb, psi_hat) for xb in np.asarray(x, dtype=np.float64)]
    c = np.stack(outs)
    return c.real.copy(), float(np.max(np.abs(c.imag))) if c.size else 0.0


def reconstruct_batch(c: np.ndarray, psi_hat: np.ndarray, adjoint_only=False):
    """[B, K, N, M] real -> ([B, N, M] real part, max |imag|)."""
    fn = adjoint if adjoint_only else reconstruct
    outs = [fn(cb, psi_hat) for cb in np.asarray(c, dtype=np.float64)]
    r = np.stack(outs)
    return r.real.copy(), float(np.max(np.abs(r.imag))) if r.size else 0.0


# ------------------------------------------------------ natural-order form
def centred_to_natural(psi_hat: np.ndarray) -> np.ndarray:
    """G_i = ifftshift(conj(psi_hat_i)): the filter as it multiplies fft2(f)."""
    return itfftshift(np.conj(np.asarray(psi_hat)))


def decompose_natural(f: np.ndarray, G: np.ndarray) -> np.ndarray:
    """c_i = ifft2(fft2(f) * G_i), any N and M."""
    X = np.fft.fft2(np.asarray(f, dtype=np.complex128))
    return np.fft.ifft2(X[None] * G, axes=(-2, -1))


def reconstruct_natural(c: np.ndarray, G: np.ndarray, weights=True):
    """ifft2(sum_i conj(G_i) fft2(c_i) [/ W]), any N and M."""
    acc = np.sum(np.conj(G) * np.fft.fft2(c, axes=(-2, -1)), axis=0)
    if weights:
        acc = acc / np.sum(np.abs(G) ** 2, axis=0)
    return np.fft.ifft2(acc)


# ------------------------------------------------- brute-force definitions
def dft2_direct(f: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT written out as its double sum (tiny inputs)."""
    f = np.asarray(f, dtype=np.complex128)
    N, M = f.shape
    ky = np.arange(N)[:, None]
    kx = np.arange(M)[:, None]
    Ey = np.exp(-2j * np.pi * ky * np.arange(N)[None, :] / N)
    Ex = np.exp(-2j * np.pi * kx * np.arange(M)[None, :] / M)
    out = np.zeros((N, M), dtype=np.complex128)
    for a in range(N):
        for b in range(M):
            out[a, b] = np.sum(f * Ey[a][:, None] * Ex[b][None, :])
    return out


def correlate_direct(f: np.ndarray, psi_centre: np.ndarray) -> np.ndarray:
    """Circular correlation c(m) = sum_n f(n + m) conj(psi(n)).

    ``psi_centre[n]`` holds the filter at centred coordinate n (index 0 is
    the filter's centre, negative coordinates wrap).  This is Def. 2.6's
    ``conj(psi^d) * f`` sampled on the full grid, written as a plain double
    loop over the translation m; the oracle's Fourier-domain decomposition
    must equal it.
    """
    f = np.asarray(f, dtype=np.complex128)
    N, M = f.shape
    out = np.zeros((N, M), dtype=np.complex128)
    pc = np.conj(np.asarray(psi_centre, dtype=np.complex128))
    for m1 in range(N):
        for m2 in range(M):
            shifted = np.roll(np.roll(f, -m1, axis=0), -m2, axis=1)
            out[m1, m2] = np.sum(shifted * pc)
    return out
