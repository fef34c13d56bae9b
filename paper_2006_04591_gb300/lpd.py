"""Learned primal-dual CT reconstruction in the image and in the shearlet
domain (Sec. 4.4, Algorithm 2).

Forward operator: the parallel-beam ray transform R of ``csrc/ray.cu`` at 30
angles (Sec. 4.4: "full angle, low-dose, 30 angles").  Iteration i = 1..I
(I = 10) with primal memory f in X^Np and dual memory h in Y^Nd
(Np = Nd = 5):

  h <- h + Gamma_i([h, T(f^(2)), g])        dual net:   Nd + 2 -> 32 -> 32 -> Nd
  f <- f + Lambda_i([f, T^*(h^(1))])         primal net: Np + 1 -> 32 -> 32 -> Np

each net being Id + W3 A W2 A W1 with 3 x 3 convolutions W and PReLU A, and
the result f^(1) after the last iteration.  In the image domain T = R / ||R||.
In the shearlet domain every primal slot holds the K shearlet coefficients
of an image as K channels ("each shearlet slice as a channel"), T =
R SH^-1 / ||R SH^-1|| with SH^-1 the reconstruction of Sec. 3.4, its adjoint
the dual-weighted decomposition of the back-projection, the primal net
(Np + 1) K -> 32 -> 32 -> Np K, and the image SH^-1 f^(1).

Readings (the paper gives the architecture but not the data protocol):
* training objects: ``synth.random_ellipses`` phantoms, 128 x 128;
* data: g = R f + e, e white Gaussian with standard deviation 5 % of the
  mean |R f| of that object ("low dose");
* f_0 = 0, h_0 = 0; loss: mean squared error against the object; Adam
  (beta2 = 0.99), learning rate 1e-3 with cosine decay, the gradient's
  global norm clipped to 1, batch 4;
* test object: the modified Shepp-Logan phantom, PSNR with peak 1 and SSIM
  (Wang et al. 2004: 11 x 11 Gaussian window, sigma 1.5, K1 = 0.01,
  K2 = 0.03, data range 1), evaluated in float64 on the host.

All convolutions, activations, the residual additions, the loss, Adam, the
ray transform and the shearlet transforms run in this package's kernels;
PyTorch holds the tensors, concatenates channels and records the graph.

    python -m paper_2006_04591_gb300.lpd [--steps S] [--out results/lpd_128.json]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import nn as NN
from . import synth
from .autograd import shearlet_dec_dual, shearlet_rec
from .ray import RayTransform, ray_adjoint, ray_forward
from .shearlet import Bank


class _Prox(torch.nn.Module):
    """Id + W3 A W2 A W1 on [B, cin, H, W]; the identity acts on the first
    cout input channels (the memory being updated)."""

    def __init__(self, cin, cout, ch, gen, device, tc):
        super().__init__()
        self.cout, self.tc = cout, tc
        dims = [cin, ch, ch, cout]
        for l in range(3):
            std = math.sqrt(2.0 / (dims[l] * 9)) * (0.1 if l == 2 else 1.0)
            w = torch.randn((dims[l + 1], dims[l], 3, 3), generator=gen) * std
            setattr(self, "w%d" % l, torch.nn.Parameter(w.to(device)))
            setattr(self, "b%d" % l, torch.nn.Parameter(torch.zeros(dims[l + 1], device=device)))
        self.a0 = torch.nn.Parameter(torch.full((1,), 0.25, device=device))
        self.a1 = torch.nn.Parameter(torch.full((1,), 0.25, device=device))

    def forward(self, x, mem):
        h = NN.prelu(NN.conv3x3(x, self.w0, self.b0, self.tc), self.a0)
        h = NN.prelu(NN.conv3x3(h, self.w1, self.b1, self.tc), self.a1)
        return NN._ResidualAdd.apply(mem, NN.conv3x3(h, self.w2, self.b2, self.tc))


class LPD(torch.nn.Module):
    """Algorithm 2 of Sec. 4.4 with ``I`` unrolled iterations.

    domain "image": primal memory [B, Np, N, N]; domain "shearlet": primal
    memory [B, Np K, N, N] (slot j = channels j K .. j K + K - 1).
    """

    def __init__(self, op: RayTransform, domain="image", bank: Bank | None = None, iters=10,
                 n_primal=5, n_dual=5, ch=32, seed=0, device="cuda", tc=True, scale=None):
        super().__init__()
        self.op, self.domain, self.bank = op, domain, bank
        self.I, self.Np, self.Nd = iters, n_primal, n_dual
        self.K = bank.K if domain == "shearlet" else 1
        gen = torch.Generator().manual_seed(seed)
        P = self.Np * self.K
        self.primal = torch.nn.ModuleList(
            [_Prox(P + self.K, P, ch, gen, device, tc) for _ in range(iters)])
        self.dual = torch.nn.ModuleList(
            [_Prox(self.Nd + 2, self.Nd, ch, gen, device, tc) for _ in range(iters)])
        self.scale = float(scale) if scale is not None else 1.0 / self._op_norm()

    # ----------------------------------------------------------- operators
    def T(self, x):
        """Primal slot [B, K, N, N] (K = 1: image) -> sinogram [B, 1, A, D]."""
        img = shearlet_rec(x, self.bank) if self.domain == "shearlet" else x[:, 0]
        return NN._Scale.apply(ray_forward(img.contiguous(), self.op), self.scale)[:, None]

    def T_adj(self, y):
        """Sinogram [B, 1, A, D] -> primal slot [B, K, N, N]."""
        img = ray_adjoint(y[:, 0].contiguous(), self.op)
        x = shearlet_dec_dual(img, self.bank) if self.domain == "shearlet" else img[:, None]
        return NN._Scale.apply(x, self.scale)

    @torch.no_grad()
    def _op_norm(self, iters=40):
        """||R|| or ||R SH^-1|| by power iteration on T^* T (unscaled)."""
        self.scale = 1.0
        g = torch.Generator(device="cuda").manual_seed(1)
        x = torch.rand((1, self.K, self.op.n, self.op.n), device="cuda", generator=g)
        lam = 1.0
        for _ in range(iters):
            y = self.T_adj(self.T(x))
            lam = y.norm().item()
            x = y / lam
        return math.sqrt(lam)

    # ------------------------------------------------------------- forward
    def forward(self, g):
        """g [B, A, D] -> reconstruction [B, N, N]."""
        B, K, N = g.shape[0], self.K, self.op.n
        gs = NN._Scale.apply(g.contiguous(), self.scale)[:, None]
        f = torch.zeros((B, self.Np * K, N, N), device=g.device)
        h = torch.zeros((B, self.Nd, self.op.n_angles, self.op.n_det), device=g.device)
        for i in range(self.I):
            h = self.dual[i](torch.cat([h, self.T(f[:, K:2 * K]), gs], dim=1), h)
            f = self.primal[i](torch.cat([f, self.T_adj(h[:, 0:1])], dim=1), f)
        first = f[:, 0:K].contiguous()
        return shearlet_rec(first, self.bank) if self.domain == "shearlet" else first[:, 0]


# -------------------------------------------------------------------- data
def phantoms(n_obj, N, seed0):
    return np.stack([synth.ellipse_phantom(synth.random_ellipses(seed0 + s), N)
                     for s in range(n_obj)]).astype(np.float32)


def noisy_data(op: RayTransform, f, gen, level=0.05):
    """g = R f + e, e ~ N(0, (level * mean |R f|)^2) per object."""
    with torch.no_grad():
        p = op.forward(f)
        sd = level * p.abs().mean(dim=(1, 2), keepdim=True)
        return p + sd * torch.randn(p.shape, device=p.device, generator=gen)


def psnr(x, ref):
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return 10.0 * math.log10(1.0 / mse)


def ssim(x, ref, data_range=1.0):
    """Mean SSIM with an 11 x 11 Gaussian window (sigma 1.5), float64."""
    from scipy.ndimage import gaussian_filter
    x, y = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    f = lambda a: gaussian_filter(a, 1.5, truncate=3.5, mode="constant")
    mx, my = f(x), f(y)
    sxx, syy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(m[5:-5, 5:-5].mean())


# ---------------------------------------------------------------- training
def resume_meta(checkpoint, domain, N, A, scales):
    """Metadata of an existing checkpoint that may be resumed by a run with
    these settings; ValueError if it was written for another network."""
    meta = torch.load(checkpoint, map_location="cpu", weights_only=False).get("meta", {})
    want = {"domain": domain, "size": N, "angles": A, "scales": scales}
    got = {k: meta.get(k) for k in want}
    if got != want:
        raise ValueError("checkpoint %s was written for %s, not %s" % (checkpoint, got, want))
    return meta


def cosine_lr(lr, it, sched_steps):
    """Cosine decay of the learning rate over sched_steps (held at the end)."""
    return 0.5 * lr * (1.0 + math.cos(math.pi * min(it, sched_steps) / sched_steps))


class _GraphStep:
    """Forward and backward of one training step captured in a CUDA graph.

    The step issues about a thousand kernel launches from Python (ten
    unrolled iterations of two three-layer networks, the ray transform and
    the shearlet transforms, forward and backward), so replaying them as one
    graph removes the per-launch host cost.  The batch is copied into static
    input buffers before each replay; the gradients the graph writes stay in
    the tensors autograd allocated during capture, which are handed back to
    the parameters before the (eager) clipping and Adam update, since
    clipping may rebind ``p.grad``.  Every kernel of the step is
    deterministic, so a replay computes what the eager step would.  No
    autograd graph of an earlier step may be alive at capture: its gradient
    accumulators keep the stream they were made on."""

    def __init__(self, net, params, g, f_true):
        self.params = params
        self.g = g.clone()
        self.f = f_true.clone()
        for p in params:
            p.grad = None
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self.loss = NN.mse(net(self.g), self.f)
            self.loss.backward()
        self.grads = [p.grad for p in params]

    def run(self, g, f_true):
        self.g.copy_(g)
        self.f.copy_(f_true)
        self.graph.replay()
        for p, gr in zip(self.params, self.grads):
            p.grad = gr
        return self.loss


def train(domain, steps=1000, batch=4, N=128, A=30, n_train=2000, lr=1e-3, seed=0, scales=2,
          log_every=100, checkpoint=None, ckpt_every=500, graph=True):
    """Train the ``domain`` network for ``steps`` steps.  With ``checkpoint``
    (a file path) the state is written there every ``ckpt_every`` steps and
    at the end (atomically), and an existing checkpoint is resumed:
    parameters, Adam state and step, with its learning-rate schedule (total
    steps and rate) kept, while the data stream restarts at that step's
    seeds.  A checkpoint of another domain, size, angle count or scale count
    is refused (ValueError).  ``graph``: after the first (eager) step,
    forward and backward replay as one CUDA graph (_GraphStep); the
    gradient clipping and the Adam update stay eager."""
    op = RayTransform(N, A, device=0)
    bank = Bank.create(N, N, scales, device=0) if domain == "shearlet" else None
    net = LPD(op, domain, bank, seed=seed)
    params = list(net.parameters())
    opt = NN.Adam(params, lr=lr, betas=(0.9, 0.99))
    pool = torch.from_numpy(phantoms(n_train, N, 10_000)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(seed + 7)
    rng = np.random.default_rng(seed)
    hist, t_steps = [], []
    start, sched_steps, base_lr = 0, steps, lr
    if checkpoint is not None and os.path.exists(checkpoint):
        meta = resume_meta(checkpoint, domain, N, A, scales)
        start, _ = NN.load_checkpoint(checkpoint, net, opt)
        sched_steps, base_lr = int(meta.get("steps", steps)), float(meta.get("lr", lr))
        rng = np.random.default_rng([seed, start])
        gen = torch.Generator(device="cuda").manual_seed(seed + 7 + 1000003 * start)
    meta = {"domain": domain, "size": N, "angles": A, "scales": scales, "batch": batch,
            "n_train": n_train, "seed": seed, "steps": sched_steps, "lr": base_lr}
    gstep = None
    for it in range(start, steps):
        opt.lr = cosine_lr(base_lr, it, sched_steps)
        idx = torch.from_numpy(rng.integers(0, n_train, batch)).cuda()
        f_true = pool[idx].contiguous()
        g = noisy_data(op, f_true, gen)
        if graph and gstep is None and it > start:
            # captured after one eager step; the eager step's autograd graph
            # is dropped first, so that the parameters' gradient accumulators
            # are made anew (on the capture stream) inside the capture
            loss = None
            gstep = _GraphStep(net, params, g, f_true)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if gstep is not None:
            loss = gstep.run(g, f_true)
        else:
            opt.zero_grad()
            loss = NN.mse(net(g), f_true)
            loss.backward()
        NN.clip_grad_norm(params, 1.0)
        opt.step()
        torch.cuda.synchronize()
        t_steps.append(time.perf_counter() - t0)
        if it % log_every == 0 or it == steps - 1:
            hist.append((it, float(loss.item())))
        if checkpoint is not None and ckpt_every > 0 and (it + 1) % ckpt_every == 0:
            NN.save_checkpoint(checkpoint, net, opt, step=it + 1, meta=meta)
    if checkpoint is not None:
        NN.save_checkpoint(checkpoint, net, opt, step=max(steps, start), meta=meta)
    return net, op, bank, hist, t_steps


@torch.no_grad()
def evaluate(net, op, N=128, seed=123):
    f = synth.ellipse_phantom(synth.shepp_logan(), N, supersample=4).astype(np.float32)
    ft = torch.from_numpy(f)[None].cuda()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    g = noisy_data(op, ft, gen)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = net(g)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rec = out[0].cpu().numpy()
    return {"psnr": psnr(rec, f), "ssim": ssim(rec, f), "reconstruct_ms": dt * 1e3}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--steps-image", type=int, default=None, help="overrides --steps")
    ap.add_argument("--steps-shearlet", type=int, default=None, help="overrides --steps")
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import _build
    _build.build()
    res = {"size": 128, "angles": 30, "iterations": 10, "n_primal": 5, "n_dual": 5,
           "batch": args.batch, "train_steps": args.steps, "noise": "5% of mean |Rf|"}
    steps = {"image": args.steps_image or args.steps, "shearlet": args.steps_shearlet or args.steps}
    res["train_steps"] = steps
    for domain in ("image", "shearlet"):
        net, op, bank, hist, ts = train(domain, steps=steps[domain], batch=args.batch,
                                        log_every=max(100, steps[domain] // 60))
        ev = evaluate(net, op)
        res[domain] = dict(ev, loss=hist, ms_per_train_step=1e3 * float(np.median(ts[5:])),
                           filters=bank.K if bank else None,
                           parameters=int(sum(p.numel() for p in net.parameters())))
        print(domain, json.dumps(res[domain]["psnr"]), res[domain]["ssim"],
              res[domain]["ms_per_train_step"])
    print(json.dumps({k: v for k, v in res.items()}, indent=1))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
