"""Pins for the FP64 learned primal-dual oracle (Sec. 4.4, Algorithm 2), CPU.

With hand-set proximal networks that are linear (PReLU slope 1, centre-tap
convolutions) Algorithm 2 reduces to the plain linear primal-dual recursion
  h_i = h_{i-1} + T f_{i-1} - s g,   f_i = f_{i-1} - tau T^* h_i,
which is written out here with the oracle's ray transform and shearlet
transforms directly.  This pins the wiring of the oracle network: which
memory slot feeds T, the channel order of the concatenations, the residual
updates, the scale and the final reconstruction.
"""

import numpy as np
import pytest
import torch

from oracle import bank as Bk
from oracle import lpd as OL
from oracle import ray as OR
from oracle import transform as OT

F64 = torch.float64


def _centre(co, ci, pairs):
    """3x3 conv weights with only centre taps: pairs of (out, in, value)."""
    w = torch.zeros((co, ci, 3, 3), dtype=F64)
    for o, i, v in pairs:
        w[o, i, 1, 1] = v
    return w


def _linear_nets(K, n_p, n_d, tau, iters):
    """Proximal nets whose output is (dual) T f^(2) - s g on every dual slot,
    (primal) -tau T^* h^(1) on every primal slot; hidden width = outputs."""
    one = torch.ones(1, dtype=F64)
    dual = []
    cd = n_d                                    # hidden width of the dual net
    for _ in range(iters):
        # dual input channels: [h (n_d), T f2 (1), s g (1)]
        w0 = _centre(cd, n_d + 2, [(o, n_d, 1.0) for o in range(cd)] +
                     [(o, n_d + 1, -1.0) for o in range(cd)])
        dual.append({"w0": w0, "b0": torch.zeros(cd, dtype=F64), "a0": one,
                     "w1": _centre(cd, cd, [(o, o, 1.0) for o in range(cd)]),
                     "b1": torch.zeros(cd, dtype=F64), "a1": one,
                     "w2": _centre(n_d, cd, [(o, o, 1.0) for o in range(n_d)]),
                     "b2": torch.zeros(n_d, dtype=F64)})
    primal = []
    cp = n_p * K
    for _ in range(iters):
        # primal input channels: [f (n_p K), T^* h1 (K)]
        w0 = _centre(cp, (n_p + 1) * K, [(j * K + k, n_p * K + k, -tau)
                                         for j in range(n_p) for k in range(K)])
        primal.append({"w0": w0, "b0": torch.zeros(cp, dtype=F64), "a0": one,
                       "w1": _centre(cp, cp, [(o, o, 1.0) for o in range(cp)]),
                       "b1": torch.zeros(cp, dtype=F64), "a1": one,
                       "w2": _centre(cp, cp, [(o, o, 1.0) for o in range(cp)]),
                       "b2": torch.zeros(cp, dtype=F64)})
    return primal, dual


@pytest.mark.parametrize("domain", ["image", "shearlet"])
def test_linear_nets_reduce_to_primal_dual_recursion(domain):
    N, A, D, iters, tau, s = 16, 6, 23, 4, 0.3, 0.8
    G = Bk.shearlet_bank(N, N, 1)["spectra"] if domain == "shearlet" else None
    K = 1 if G is None else G.shape[0]
    op = OL.Operator(N, A, D, G=G, scale=s)
    g = np.random.default_rng(0).standard_normal((2, A, D))
    primal, dual = _linear_nets(K, 2, 2, tau, iters)
    got = OL.lpd(torch.as_tensor(g), op, primal, dual, 2, 2).numpy()
    # the recursion, written with the oracle transforms (numpy)
    W = None if G is None else np.sum(G ** 2, axis=0)
    rec = (lambda c: c[:, 0]) if G is None else \
        (lambda c: np.stack([OT.reconstruct_natural(cb, G).real for cb in c]))
    dual_dec = (lambda x: x[:, None]) if G is None else \
        (lambda x: np.stack([OT.decompose_natural(xb, G / W).real for xb in x]))
    f = np.zeros((2, K, N, N))
    h = np.zeros((2, A, D))
    for _ in range(iters):
        h = h + s * OR.forward(rec(f), A, D) - s * g
        f = f - tau * s * dual_dec(OR.adjoint(h, N))
    want = rec(f)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_power_iteration_norm_matches_svd():
    import scipy.sparse.linalg as sla
    op = OL.Operator(24, 9, 35)
    want = sla.svds(OR.system_matrix(24, 9, 35), k=1, return_singular_vectors=False)[0]
    assert abs(OL.op_norm(op) - want) <= 1e-9 * want
