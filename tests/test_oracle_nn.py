"""Pins for the learned-part oracle (CPU): convolution against the library
routine torch.nn.functional.conv2d, gradients against finite differences,
the gate's limit, PReLU's two branches, Adam against its closed form."""

import numpy as np
import torch

from oracle import nn as ON


def test_conv_matches_library_conv2d():
    g = torch.Generator().manual_seed(0)
    x = torch.randn((2, 3, 9, 7), generator=g, dtype=torch.float64)
    w = torch.randn((4, 3, 3, 3), generator=g, dtype=torch.float64)
    b = torch.randn(4, generator=g, dtype=torch.float64)
    ref = torch.nn.functional.conv2d(x, w, b, padding=1)
    assert torch.allclose(ON.conv3x3(x, w, b), ref, atol=1e-12)


def test_gradients_match_finite_differences():
    g = torch.Generator().manual_seed(1)
    x = torch.randn((2, 2, 8, 8), generator=g, dtype=torch.float64)
    params = {"w0": torch.randn((3, 2, 3, 3), generator=g, dtype=torch.float64),
              "b0": torch.randn(3, generator=g, dtype=torch.float64),
              "a0": torch.tensor(0.25, dtype=torch.float64)}
    for p in params.values():
        p.requires_grad_(True)

    def f():
        h = ON.prelu(ON.conv3x3(x, params["w0"], params["b0"]), params["a0"])
        return (h ** 2).sum()
    f().backward()
    eps = 1e-6
    for name in ("w0", "b0", "a0"):
        p = params[name]
        flat = p.detach().reshape(-1)
        for idx in range(min(4, flat.numel())):
            with torch.no_grad():
                orig = flat[idx].item()
                flat[idx] = orig + eps
                fp = f().item()
                flat[idx] = orig - eps
                fm = f().item()
                flat[idx] = orig
            fd = (fp - fm) / (2 * eps)
            assert abs(fd - p.grad.reshape(-1)[idx].item()) <= 1e-6 * max(1, abs(fd))


def test_prelu_branches_and_softplus():
    x = torch.tensor([-2.0, -0.5, 0.0, 0.5, 2.0], dtype=torch.float64)
    assert torch.equal(ON.prelu(x, 0.1), torch.tensor([-0.2, -0.05, 0.0, 0.5, 2.0], dtype=torch.float64))
    assert torch.allclose(ON.softplus(x), torch.log(1 + torch.exp(x)), atol=1e-15)


def test_gate_tends_to_hard_threshold():
    c = torch.tensor([[[[-1.0, -0.3, 0.2, 0.6, 2.0]]]], dtype=torch.float64)
    d = torch.tensor([[0.5]], dtype=torch.float64)
    hard = torch.where(c.abs() >= 0.5, c, torch.zeros_like(c))
    assert torch.allclose(ON.gate(c, d, 1e-4), hard, atol=1e-12)


def test_torch_transforms_match_numpy_oracle():
    from oracle import bank as Bk
    from oracle import transform as T
    b = Bk.shearlet_bank(32, 32, 2)
    G = torch.as_tensor(b["spectra"])
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 32, 32))
    c = ON.dec_t(torch.as_tensor(x), G)
    want, _ = T.decompose_batch(x, b["psi_hat"])
    assert np.abs(c.numpy() - want).max() < 1e-12
    r = ON.rec_t(c, G)
    assert np.abs(r.numpy() - x).max() < 1e-12


def test_adam_first_step_is_sign_times_lr():
    p = torch.tensor([1.0, -2.0, 3.0], dtype=torch.float64)
    g = torch.tensor([0.5, -4.0, 1e-3], dtype=torch.float64)
    p1, m, v = ON.adam_step(p, g, torch.zeros(3, dtype=torch.float64),
                            torch.zeros(3, dtype=torch.float64), 1, 0.01, eps=0.0)
    assert torch.allclose(p1, p - 0.01 * torch.sign(g), atol=1e-15)


def test_avgpool_and_gap():
    x = torch.arange(16, dtype=torch.float64).reshape(1, 1, 4, 4)
    assert torch.equal(ON.avgpool(x, 2)[0, 0], torch.tensor([[2.5, 4.5], [10.5, 12.5]], dtype=torch.float64))
    assert ON.gap(x).item() == 7.5
