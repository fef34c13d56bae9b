"""FP64 oracle of the learned primal-dual reconstruction (Sec. 4.4,
Algorithm 2), image and shearlet domain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain float64 torch CPU definitions (gradients by torch's autograd):

* T = s R (image domain) or s R SH^-1 (shearlet domain), with R the sparse
  system matrix of ``oracle.ray``, SH^-1 the reconstruction of Sec. 3.4
  (``oracle.nn.rec_t``) and s a given scale; T^* = s R^T, or
  s SH^-* R^T with SH^-* the decomposition with G_i / W (the adjoint of the
  reconstruction);
* each learned proximal is Id + W3 A W2 A W1 (3 x 3 convolutions, PReLU)
  acting on the memory it updates;
* iteration i: h <- h + Gamma_i([h, T(f^(2)), s g]);
  f <- f + Lambda_i([f, T^*(h^(1))]); the result is f^(1) (through SH^-1 in
  the shearlet domain), with f_0 = 0 and h_0 = 0.
"""

from __future__ import annotations

import numpy as np
import torch

from . import nn as ON
from . import ray as OR

F64 = torch.float64


class Operator:
    def __init__(self, N, A, D, G=None, scale=1.0):
        M = OR.system_matrix(N, A, D).tocoo()
        self.M = torch.sparse_coo_tensor(np.vstack([M.row, M.col]), M.data, M.shape, dtype=F64,
                                         check_invariants=True)
        self.MT = self.M.t().coalesce()
        self.N, self.A, self.D, self.scale = N, A, D, float(scale)
        self.G = None if G is None else torch.as_tensor(np.asarray(G), dtype=F64)

    def R(self, img):                 # [B, N, N] -> [B, A, D]
        B = img.shape[0]
        return torch.sparse.mm(self.M, img.reshape(B, -1).T).T.reshape(B, self.A, self.D)

    def RT(self, y):                  # [B, A, D] -> [B, N, N]
        B = y.shape[0]
        return torch.sparse.mm(self.MT, y.reshape(B, -1).T).T.reshape(B, self.N, self.N)

    def T(self, x):                   # [B, K, N, N] -> [B, 1, A, D]
        img = ON.rec_t(x, self.G) if self.G is not None else x[:, 0]
        return (self.scale * self.R(img))[:, None]

    def T_adj(self, y):               # [B, 1, A, D] -> [B, K, N, N]
        img = self.RT(y[:, 0])
        if self.G is None:
            return self.scale * img[:, None]
        W = torch.sum(self.G ** 2, dim=0)
        return self.scale * ON.dec_t(img, self.G / W[None])


def prox(x, mem, p):
    h = ON.prelu(ON.conv3x3(x, p["w0"], p["b0"]), p["a0"])
    h = ON.prelu(ON.conv3x3(h, p["w1"], p["b1"]), p["a1"])
    return mem + ON.conv3x3(h, p["w2"], p["b2"])


def lpd(g, op: Operator, primal, dual, n_primal, n_dual):
    """g [B, A, D] -> [B, N, N]; primal / dual: lists of parameter dicts."""
    B = g.shape[0]
    K = 1 if op.G is None else op.G.shape[0]
    f = torch.zeros((B, n_primal * K, op.N, op.N), dtype=F64)
    h = torch.zeros((B, n_dual, op.A, op.D), dtype=F64)
    gs = (op.scale * g)[:, None]
    for pp, pd in zip(primal, dual):
        h = prox(torch.cat([h, op.T(f[:, K:2 * K]), gs], dim=1), h, pd)
        f = prox(torch.cat([f, op.T_adj(h[:, 0:1])], dim=1), f, pp)
    first = f[:, 0:K]
    return ON.rec_t(first, op.G) if op.G is not None else first[:, 0]


def op_norm(op: Operator, iters=200, seed=0):
    """||T|| (with scale 1) by float64 power iteration on T^* T."""
    s = op.scale
    op.scale = 1.0
    K = 1 if op.G is None else op.G.shape[0]
    x = torch.as_tensor(np.random.default_rng(seed).random((1, K, op.N, op.N)), dtype=F64)
    lam = 1.0
    for _ in range(iters):
        y = op.T_adj(op.T(x))
        lam = float(torch.linalg.vector_norm(y))
        x = y / lam
    op.scale = s
    return float(np.sqrt(lam))
