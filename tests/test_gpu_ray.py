"""GPU parity of the ray transform (``csrc/ray.cu``) against the FP64 oracle
(``oracle/ray.py``): forward and adjoint element by element, the adjoint
identity, and the exact line integrals of ellipses through the GPU path.

Tolerance (derived from the arithmetic): the kernels evaluate the sample
position u = A d + B t + C in float32, |u| <= about 1.5 n, so u carries an
error of about 2e-7 n pixel widths; through the linear interpolation and
the n samples of weight <= 2.9/n this bounds the error of a ray sum by about
1e-6 n max|f|.  The tests allow 1e-6 n max|f| + 1e-6 max|p|.
"""

import numpy as np
import pytest

from oracle import ray as R
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(16, 1, 23), (37, 7, 53), (64, 30, 91), (128, 30, 182), (96, 45, 64), (50, 3, 300)]


def _op(n, A, D):
    from paper_2006_04591_gb300.ray import RayTransform
    return RayTransform(n, A, D, device=0)


@pytest.mark.parametrize("n,A,D", CASES)
def test_forward_and_adjoint_parity(n, A, D):
    op = _op(n, A, D)
    rng = np.random.default_rng(n + A)
    f = np.stack([synth.ellipse_phantom(synth.random_ellipses(s), n) for s in range(2)] +
                 [rng.standard_normal((n, n))]).astype(np.float32)
    p = op.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    want = R.forward(f, A, D)
    for b in range(3):
        tol = 1e-6 * n * np.abs(f[b]).max() + 1e-6 * np.abs(want[b]).max()
        assert np.abs(p[b] - want[b]).max() <= tol, (b, np.abs(p[b] - want[b]).max(), tol)
    y = rng.standard_normal((2, A, D)).astype(np.float32)
    g = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    want = R.adjoint(y, n)
    for b in range(2):
        tol = 1e-6 * n * np.abs(y[b]).max() * (2.9 / n) * 3 * A + 1e-6 * np.abs(want[b]).max()
        assert np.abs(g[b] - want[b]).max() <= tol, (b, np.abs(g[b] - want[b]).max(), tol)


@pytest.mark.parametrize("n,A,D", CASES[2:4])
def test_adjoint_identity_on_gpu(n, A, D):
    op = _op(n, A, D)
    gen = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn((4, n, n), device="cuda", generator=gen)
    y = torch.randn((4, A, D), device="cuda", generator=gen)
    lhs = (op.forward(x).double() * y.double()).sum().item()
    rhs = (x.double() * op.adjoint(y).double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_shepp_logan_line_integrals():
    n, A, D = 256, 30, 363
    op = _op(n, A, D)
    tab = synth.shepp_logan()
    f = synth.ellipse_phantom(tab, n, supersample=8, clip=False).astype(np.float32)
    p = op.forward(torch.from_numpy(f)[None].cuda())[0].cpu().numpy()
    exact = R.ellipse_sinogram(tab, A, D)
    assert np.linalg.norm(p - exact) / np.linalg.norm(exact) < 0.02


def test_autograd_and_norm():
    from paper_2006_04591_gb300.ray import ray_adjoint, ray_forward
    n, A, D = 64, 30, 91
    op = _op(n, A, D)
    x = torch.randn((2, n, n), device="cuda", requires_grad=True)
    y = torch.randn((2, A, D), device="cuda")
    (ray_forward(x, op) * y).sum().backward()
    assert torch.allclose(x.grad, op.adjoint(y), rtol=0, atol=1e-6)
    y2 = y.clone().requires_grad_(True)
    (ray_adjoint(y2, op) * x.detach()).sum().backward()
    assert torch.allclose(y2.grad, op.forward(x.detach()), rtol=0, atol=1e-6)
    # ||R|| against the oracle's matrix 2-norm
    import scipy.sparse.linalg as sla
    want = sla.svds(R.system_matrix(n, A, D), k=1, return_singular_vectors=False)[0]
    assert abs(op.norm(60) - want) <= 1e-3 * want


def test_rejects_bad_arguments():
    from paper_2006_04591_gb300.ray import RayTransform
    from paper_2006_04591_gb300.shearlet import ShearletError
    with pytest.raises(ShearletError):
        RayTransform(1, 30, 10)
    op = _op(16, 4, 23)
    with pytest.raises(ValueError):
        op.forward(torch.zeros((1, 15, 16), device="cuda"))
    assert op.forward(torch.zeros((0, 16, 16), device="cuda")).shape == (0, 4, 23)
