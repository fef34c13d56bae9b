"""FP64 oracle: the discrete parallel-beam ray transform of Sec. 4.4.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4.4 defines the Radon transform as the line integral
``R f(s, phi) = int f(s theta + t theta_perp) dt`` with
``theta = (cos phi, sin phi)`` and ``theta_perp = (-sin phi, cos phi)``, and
measures it at 30 angles over the full half-turn.  The paper computes it with
ODL / ASTRA, which are not available; the discretisation is therefore a
reading, stated here and written out as an explicit sparse system matrix so
that the adjoint is its transpose by construction.

Geometry (reading):
* the image f[i, j] (row i, column j) covers the square [-1, 1]^2 with
  N x N pixels of side h = 2/N; pixel (i, j) has centre
  (x_j, y_i) = (-1 + (j + 1/2) h, -1 + (i + 1/2) h), row index = y;
* angles phi_a = pi a / A, a = 0..A-1;
* detector bins s_d = -S + (d + 1/2) ds, S = sqrt(2), ds = 2 S / D,
  d = 0..D-1 (the bins cover the projection of the whole square).

Discretisation (Joseph's method): the line x cos(phi) + y sin(phi) = s is
sampled once per pixel row when |cos phi| >= |sin phi| (x found from y) and
once per pixel column otherwise (y found from x); at each sample the image
is interpolated linearly between the two neighbouring pixels of that row or
column (zero outside the image), and the samples are summed with the path
length per row, h / |cos phi| (per column, h / |sin phi|).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

S_MAX = float(np.sqrt(2.0))


def geometry(N: int, A: int, D: int) -> dict:
    """Pixel centres, angles and detector bin centres of the reading above."""
    h = 2.0 / N
    return {
        "h": h,
        "x": -1.0 + (np.arange(N) + 0.5) * h,       # column centres
        "y": -1.0 + (np.arange(N) + 0.5) * h,       # row centres
        "phi": np.pi * np.arange(A) / A,
        "s": -S_MAX + (np.arange(D) + 0.5) * (2.0 * S_MAX / D),
    }


def system_matrix(N: int, A: int, D: int) -> sp.csr_matrix:
    """Sparse [A*D, N*N] matrix of the discrete transform (row a*D + d is the
    ray (phi_a, s_d), column i*N + j the pixel (i, j))."""
    g = geometry(N, A, D)
    h = g["h"]
    rows, cols, vals = [], [], []
    d = np.arange(D)[:, None]
    t = np.arange(N)[None, :]                    # sample index: row or column
    for a, phi in enumerate(g["phi"]):
        c, s_ = np.cos(phi), np.sin(phi)
        by_rows = abs(c) >= abs(s_)
        step = h / (abs(c) if by_rows else abs(s_))
        s = g["s"][:, None]
        if by_rows:                              # sample on row t: x from y_t
            u = ((s - g["y"][None, :] * s_) / c + 1.0) / h - 0.5
        else:                                    # sample on column t: y from x_t
            u = ((s - g["x"][None, :] * c) / s_ + 1.0) / h - 0.5
        k0 = np.floor(u).astype(np.int64)
        w = u - k0
        for k, wk in ((k0, 1.0 - w), (k0 + 1, w)):
            ok = (k >= 0) & (k < N) & (wk != 0.0)
            kk = np.where(ok, k, 0)
            pix = t * N + kk if by_rows else kk * N + t
            rr = np.broadcast_to(a * D + d, k.shape)
            rows.append(rr[ok])
            cols.append(np.broadcast_to(pix, k.shape)[ok])
            vals.append(wk[ok] * step)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(A * D, N * N))


_CACHE: dict = {}


def _matrix(N, A, D):
    key = (N, A, D)
    if key not in _CACHE:
        _CACHE[key] = system_matrix(N, A, D)
    return _CACHE[key]


def forward(f: np.ndarray, A: int, D: int) -> np.ndarray:
    """[..., N, N] images -> [..., A, D] sinograms."""
    f = np.asarray(f, np.float64)
    N = f.shape[-1]
    M = _matrix(N, A, D)
    flat = f.reshape(-1, N * N)
    return (M @ flat.T).T.reshape(f.shape[:-2] + (A, D))


def adjoint(p: np.ndarray, N: int) -> np.ndarray:
    """[..., A, D] sinograms -> [..., N, N] images (the transpose)."""
    p = np.asarray(p, np.float64)
    A, D = p.shape[-2:]
    M = _matrix(N, A, D)
    flat = p.reshape(-1, A * D)
    return (M.T @ flat.T).T.reshape(p.shape[:-2] + (N, N))


# ------------------------------------------------------ analytic ellipses
def ellipse_sinogram(ellipses, A: int, D: int) -> np.ndarray:
    """Exact line integrals of a sum of filled ellipses at the bins above.

    ``ellipses``: rows (value, a, b, x0, y0, alpha) -- semi-axis a along the
    direction alpha, b across it, centre (x0, y0).  For one ellipse the line
    x . theta = s cuts a chord of length 2 a b sqrt(r^2 - s'^2) / r^2, with
    s' = s - (x0, y0) . theta and r^2 = a^2 cos^2(phi - alpha) +
    b^2 sin^2(phi - alpha) (the support function squared), zero for
    |s'| >= r.
    """
    g = geometry(1, A, D)
    phi = g["phi"][:, None]
    s = g["s"][None, :]
    out = np.zeros((A, D))
    for val, a, b, x0, y0, alpha in np.asarray(ellipses, np.float64):
        sp_ = s - (x0 * np.cos(phi) + y0 * np.sin(phi))
        r2 = a * a * np.cos(phi - alpha) ** 2 + b * b * np.sin(phi - alpha) ** 2
        inside = sp_ * sp_ < r2
        chord = np.where(inside, 2.0 * a * b * np.sqrt(np.maximum(r2 - sp_ * sp_, 0.0)) / r2, 0.0)
        out += val * chord
    return out


def ellipse_image(ellipses, N: int, supersample: int = 4) -> np.ndarray:
    """Pixel averages of a sum of filled ellipses on the grid above
    (supersample^2 point samples per pixel)."""
    h = 2.0 / N
    q = (np.arange(N * supersample) + 0.5) * (h / supersample) - 1.0
    Y, X = np.meshgrid(q, q, indexing="ij")
    img = np.zeros_like(X)
    for val, a, b, x0, y0, alpha in np.asarray(ellipses, np.float64):
        ca, sa = np.cos(alpha), np.sin(alpha)
        u = (X - x0) * ca + (Y - y0) * sa
        v = -(X - x0) * sa + (Y - y0) * ca
        img += val * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    return img.reshape(N, supersample, N, supersample).mean(axis=(1, 3))
