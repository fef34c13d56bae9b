"""Learned per-subband thresholds for shearlet inpainting, and the
coefficient-domain network step.

Inpainting (Sec. 4.3, Alg. "Shearlet inpainting by iterative hard
thresholding") runs T iterations of f <- SH^{-1} T_delta SH (M (f_m - f) + f)
with thresholds delta_t RMS_i.  The plain method decays delta geometrically
over 60 iterations.  Here a small CNN (ThresholdNet) looks at [f_masked, mask]
and predicts all thresholds delta_{t,i} (t < 10, i < K) of a 10-iteration
loop.  Training unrolls the 10 iterations with a relaxed threshold
c sigmoid((|c| / delta - 1) / tau), tau annealed towards 0, and minimises the
mean squared error to the clean image; its backward passes run through the
adjoint transforms (shl_adjoint for the decomposition, the dual-weighted
decomposition for the reconstruction) and the library's network kernels.
Inference uses the hard threshold through shl_decompose_masked and
shl_reconstruct, i.e. exactly the plain method's kernels with learned
thresholds.  The plain loop stays as fallback and as the PSNR reference.

Run ``python -m paper_2006_04591_gb300.learned`` to train on 2,000 seeded
512 x 512 pairs and compare with the plain method on 8 held-out images.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import apps, nn, synth
from .autograd import shearlet_dec, shearlet_rec
from .shearlet import SHL_OP_SHRINK, Bank


def unrolled_iht(bank: Bank, f_masked, mask_u8, deltas, tau, rms):
    """T relaxed iterations, differentiable in deltas [B, T, K] (x RMS_i)."""
    f = torch.zeros_like(f_masked)
    for t in range(deltas.shape[1]):
        u = nn.mask_mix(f_masked, mask_u8, f)
        c = shearlet_dec(u, bank)
        f = shearlet_rec(nn.gate(c, deltas[:, t].contiguous(), tau, scale=rms), bank)
    return f


def hard_iht(bank: Bank, f_masked, mask_u8, thresholds, out_each=None):
    """Hard-threshold iterations with given absolute thresholds [T, B, K]
    (one shl_shrink per iteration: the coefficients stay in registers)."""
    B = f_masked.shape[0]
    ws = bank.workspace(SHL_OP_SHRINK, B)
    f = torch.zeros_like(f_masked)
    g = torch.empty_like(f)
    for t in range(thresholds.shape[0]):
        bank.shrink(f_masked, thresholds[t], mask_u8=mask_u8, f_est=f, out=g, ws=ws)
        f, g = g, f
        if out_each is not None:
            out_each(t, f)
    return f


def _softplus_inv(y):
    return float(np.log(np.expm1(y)))


def make_net(bank: Bank, T=10, delta0=5.0, delta_min=0.02, seed=0, pool=4, ch=32):
    """ThresholdNet whose initial output is the plain geometric schedule."""
    net = nn.ThresholdNet(bank.K, T=T, ch=ch, pool=pool, seed=seed, device="cuda:%d" % bank.device)
    lam = (delta_min / delta0) ** (1.0 / max(T - 1, 1))
    with torch.no_grad():
        b = torch.tensor([_softplus_inv(delta0 * lam ** t) for t in range(T)], dtype=torch.float32)
        net.bl.copy_(b.repeat_interleave(bank.K).to(net.bl.device))
    return net


def _make_pairs(args):
    """One training batch: cartoon+texture images and Bernoulli masks (uint8)
    for the given seeds (runs in a worker process)."""
    n, p, seeds = args
    clean = np.stack([synth.cartoon_texture(n, n, int(s)) for s in seeds]).astype(np.float32)
    mask = np.stack([synth.bernoulli_mask(n, n, p, 50_000 + int(s)) for s in seeds])
    return clean, mask.astype(np.uint8)


class _Pairs:
    """Seeded (clean, mask) batches produced ahead by a pool of spawned worker
    processes (the numpy image synthesis would otherwise bound the training
    step on the host).

    The seeds of every step are drawn up front, so the training data order is
    deterministic; at most `depth` batches are in flight or waiting."""

    def __init__(self, n, seed0, n_pairs, batch, steps, p=0.5, rng_seed=0, workers=None, depth=None):
        import multiprocessing as mp
        import os
        from collections import deque
        rng = np.random.default_rng(rng_seed)
        self.seeds = seed0 + rng.integers(0, n_pairs, size=(steps, batch))
        self.n, self.p = n, p
        nw = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
        self.pool = mp.get_context("spawn").Pool(nw)
        self.pending = deque()
        self.next_submit = 0
        self.depth = depth or 2 * nw
        while self.next_submit < min(self.depth, len(self.seeds)):
            self._submit()

    def _submit(self):
        args = (self.n, self.p, self.seeds[self.next_submit])
        self.pending.append(self.pool.apply_async(_make_pairs, (args,)))
        self.next_submit += 1

    def get(self):
        res = self.pending.popleft()
        if self.next_submit < len(self.seeds):
            self._submit()
        clean, mask = res.get(timeout=600)
        return clean, mask.astype(np.float32)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def train_thresholds(bank: Bank, steps=300, batch=4, T=10, n_pairs=2000, seed0=10000, lr=2e-3,
                     tau0=0.3, tau1=0.02, delta0=5.0, log=None):
    dev = torch.device("cuda", bank.device)
    net = make_net(bank, T=T, delta0=delta0)
    opt = nn.Adam(list(net.parameters()), lr=lr)
    rms = torch.tensor(bank.rms, dtype=torch.float32, device=dev)
    pairs = _Pairs(bank.rows, seed0, n_pairs, batch, steps)
    hist = []
    try:
        for step in range(steps):
            tau = tau0 * (tau1 / tau0) ** (step / max(steps - 1, 1))
            clean, mask = pairs.get()
            fm = torch.from_numpy(clean * mask).to(dev)
            clean = torch.from_numpy(clean).to(dev)
            mu8 = torch.from_numpy(mask.astype(np.uint8)).to(dev)
            mask = torch.from_numpy(mask).to(dev)
            d = net(torch.stack([fm, mask], dim=1))
            f = unrolled_iht(bank, fm, mu8, d, tau, rms)
            loss = nn.mse(f, clean)
            opt.zero_grad()
            loss.backward()
            opt.step()
            if step % 25 == 0 or step == steps - 1:
                l = float(loss.item())
                hist.append((step, tau, l))
                if log:
                    log("step %d tau %.3f loss %.5f psnr %.2f" % (step, tau, l, -10 * math.log10(l)))
    finally:
        pairs.close()
    return net, hist


@torch.no_grad()
def learned_thresholds(bank: Bank, net, fm, mask):
    """Absolute thresholds [T, B, K] predicted by the network."""
    d = net(torch.stack([fm, mask], dim=1))                       # [B, T, K]
    rms = torch.tensor(bank.rms, dtype=torch.float32, device=fm.device)
    th = torch.empty((d.shape[1], d.shape[0], d.shape[2]), dtype=torch.float32, device=fm.device)
    nn.scale_thresholds(d, rms, th)
    return th


@torch.no_grad()
def evaluate(bank: Bank, net, B=8, seed0=2000, plain_iters=60, delta_min=0.02, repeats=3):
    """Plain 60-iteration IHT vs the learned 10-iteration loop on held-out images."""
    dev = torch.device("cuda", bank.device)
    clean, mask, masked = synth.inpaint_batch(B, bank.rows, 0.5, seed0)
    clean_t = torch.from_numpy(clean.astype(np.float32)).to(dev)
    fm = torch.from_numpy(masked.astype(np.float32)).to(dev)
    mk = torch.from_numpy(mask.astype(np.float32)).to(dev)
    mu8 = mk.to(torch.uint8)
    stream = torch.cuda.current_stream(dev)

    def plain_thresholds():
        return apps.iht_schedule(bank, fm, plain_iters, delta_min)

    # plain method: per-iteration PSNR (untimed pass) and per-iteration time (timed pass)
    psnr_plain = []
    hard_iht(bank, fm, mu8, plain_thresholds(),
             out_each=lambda t, f: psnr_plain.append(apps.psnr(f, clean_t).mean().item()))
    t_plain = []
    for _ in range(repeats):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(plain_iters + 1)]
        torch.cuda.synchronize()
        evs[0].record(stream)
        th = plain_thresholds()          # includes the start-threshold decomposition
        hard_iht(bank, fm, mu8, th, out_each=lambda t, f: evs[t + 1].record(stream))
        torch.cuda.synchronize()
        t_plain.append([evs[0].elapsed_time(e) / 1e3 for e in evs[1:]])
    t_plain = np.median(np.asarray(t_plain), axis=0)

    # learned: network + T hard iterations
    f = hard_iht(bank, fm, mu8, learned_thresholds(bank, net, fm, mk))
    p_learned = apps.psnr(f, clean_t).mean().item()
    t_learned = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        hard_iht(bank, fm, mu8, learned_thresholds(bank, net, fm, mk))
        b.record(stream)
        torch.cuda.synchronize()
        t_learned.append(a.elapsed_time(b) / 1e3)
    t_learned = float(np.median(t_learned))
    reach = [i for i, p in enumerate(psnr_plain) if p >= p_learned]
    return {
        "images": B, "size": bank.rows, "filters": bank.K, "mask": "Bernoulli(0.5)",
        "plain_iterations": plain_iters, "plain_psnr_final": psnr_plain[-1],
        "plain_seconds_total": float(t_plain[-1]),
        "plain_psnr_per_iteration": psnr_plain,
        "learned_iterations": int(net.T), "learned_psnr": p_learned,
        "learned_seconds": t_learned,
        "plain_seconds_to_learned_psnr": float(t_plain[reach[0]]) if reach else None,
        "plain_iterations_to_learned_psnr": (reach[0] + 1) if reach else None,
        "masked_psnr": apps.psnr(fm, clean_t).mean().item(),
    }


def coeff_net_step(bank: Bank, net, opt, x_noisy, clean):
    """One training step of the coefficient-domain network: bfloat16
    decomposition -> c + CNN(c) -> reconstruction -> MSE to the clean batch."""
    c16 = shearlet_dec(x_noisy, bank, torch.bfloat16)
    c = nn.bf16_to_float(c16)
    y = shearlet_rec(net(c), bank)
    loss = nn.mse(y, clean)
    opt.zero_grad()
    loss.backward()
    opt.step()
    return loss


def time_coeff_net_step(B=32, N=256, scales=3, steps=10, warmup=3, tc=True):
    """Training-step time of the coefficient network (bfloat16 coefficients;
    tc: tensor-core convolutions for the forward and input gradients)."""
    bank = Bank.create(N, N, scales, device=0)
    dev = torch.device("cuda", 0)
    clean, noisy = synth.denoise_batch(B, N, 30 / 255, seed0=1000)
    x = torch.from_numpy(noisy.astype(np.float32)).to(dev)
    y = torch.from_numpy(clean.astype(np.float32)).to(dev)
    net = nn.CoeffNet(bank.K, ch=32, seed=0, device=dev, tc=tc)
    opt = nn.Adam(list(net.parameters()), lr=1e-3)
    losses = []
    for _ in range(warmup):
        losses.append(float(coeff_net_step(bank, net, opt, x, y).item()))
    st = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(steps):
        l = coeff_net_step(bank, net, opt, x, y)
    b.record(st)
    torch.cuda.synchronize()
    losses.append(float(l.item()))
    ms = a.elapsed_time(b) / steps
    conv_flops = 2 * B * N * N * 9 * (bank.K * 32 + 32 * 32 + 32 * bank.K) * 3   # fwd + 2 bwd
    return {"batch": B, "size": N, "filters": bank.K, "coeff_dtype": "bf16",
            "conv": "tcgen05 bf16 (forward, input and weight gradients)" if tc else "float32",
            "ms_per_train_step": ms, "conv_tflops": conv_flops / (ms / 1e3) / 1e12,
            "loss_first": losses[0], "loss_last": losses[-1]}


CHECKPOINT_KIND = "threshold-net"


def checkpoint_meta(bank: Bank, net, args=None):
    """What a threshold-network checkpoint was trained for; load_threshold_net
    refuses a checkpoint whose bank or iteration count differ."""
    m = {"kind": CHECKPOINT_KIND, "size": bank.rows, "filters": bank.K, "iterations": int(net.T),
         "pool": int(net.pool), "train_pairs": 2000, "train_seeds": "10000..11999",
         "mask": "Bernoulli(0.5)"}
    if args is not None:
        m.update({"train_steps": args.steps, "train_batch": args.batch, "train_lr": args.lr})
    return m


def load_threshold_net(bank: Bank, path):
    """ThresholdNet restored from a checkpoint written by ``main --save``."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    meta = state.get("meta", {})
    if meta.get("kind") != CHECKPOINT_KIND or meta.get("size") != bank.rows or \
            meta.get("filters") != bank.K:
        raise ValueError("checkpoint %s is not a threshold network for %d x %d, K = %d"
                         % (path, bank.rows, bank.rows, bank.K))
    net = nn.ThresholdNet(bank.K, T=int(meta["iterations"]), pool=int(meta.get("pool", 4)),
                          device="cuda:%d" % bank.device)
    nn.load_checkpoint(path, net)
    return net


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--iters", type=int, default=10, help="unrolled iterations T")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--save", default=None, help="write the trained network (nn.save_checkpoint)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--coeff-net", action="store_true", help="time the coefficient-network step")
    args = ap.parse_args()
    from . import _build
    _build.build()
    if args.coeff_net:
        res = time_coeff_net_step()
        print(json.dumps(res))
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(res, fh, indent=1)
        return
    bank = Bank.create(args.size, args.size, 4, device=0)
    t0 = time.time()
    net, hist = train_thresholds(bank, steps=args.steps, batch=args.batch, T=args.iters,
                                 lr=args.lr, log=print)
    train_s = time.time() - t0
    res = evaluate(bank, net)
    res.update({"train_steps": args.steps, "train_batch": args.batch, "train_pairs": 2000,
                "train_lr": args.lr, "train_seconds": train_s, "train_history": hist})
    if args.save:
        nn.save_checkpoint(args.save, net, step=args.steps, meta=checkpoint_meta(bank, net, args))
    print(json.dumps({k: v for k, v in res.items() if k != "plain_psnr_per_iteration"}))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
