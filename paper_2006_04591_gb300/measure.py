"""Throughput of the transform at each workload's shape (CUDA-event timing).

    python -m paper_2006_04591_gb300.measure [--out results/configs.json]
    python -m paper_2006_04591_gb300.measure --case N B
    python -m paper_2006_04591_gb300.measure --general [--out FILE]

``--case N B [--bf16]`` runs only two decomposition + reconstruction passes of B
cartoon images of N x N with the 4-scale bank (49 filters): the small case
that the ncu captures under profiles/ are taken on (launch order per pass:
image R2C rows, image spectrum lines, coefficient lines, coefficient C2R
rows; then coefficient R2C rows, reconstruction lines, image C2R rows).

For every point: decomposition + reconstruction of a batch (inputs resident
on the device, L2 flushed between timed repetitions), shearlet coefficients
per second, algorithmic HBM bytes per second (images and coefficients once
per direction, float32 half-spectrum filters once per direction) and its
fraction of the measured copy bandwidth.  Also the denoising time and PSNR
at 16 x 512 x 512, the differentiable layer's forward + backward time at
32 x 256 x 256 with bfloat16 coefficients, and the filter-bank construction
time on the host and on the GPU.

``--general`` times only the general kernels (sizes that are not powers of
two, and the 512 x 512 bank forced onto them), with the per-launch-name
device times of one pass from the library's own event profile.
"""

from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import apps, synth
from .autograd import shearlet_dec, shearlet_rec
from .shearlet import SHL_OP_DECOMPOSE, SHL_OP_RECONSTRUCT, Bank

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def _time(fn, reps=10, warmup=3):
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")   # 512 MiB > L2
    for _ in range(warmup):
        fn()
    st = torch.cuda.current_stream()
    tot = 0.0
    for i in range(reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps / 1e3


def alg_bytes(B, K, N, M, s):
    H = N * (M // 2 + 1)
    return B * (4 * N * M + s * K * N * M) + 4 * K * H + B * (s * K * N * M + 4 * N * M) + 4 * K * H + 4 * H


def transform_point(bank, B, dtype, seed=5000):
    N, M, K = bank.rows, bank.cols, bank.K
    x = torch.from_numpy(np.stack([synth.cartoon(N, M, seed + b) for b in range(B)]).astype(np.float32)).cuda()
    c = torch.empty((B, K, N, M), dtype=dtype, device="cuda")
    y = torch.empty_like(x)
    wd, wr = bank.workspace(SHL_OP_DECOMPOSE, B), bank.workspace(SHL_OP_RECONSTRUCT, B)

    def step():
        bank.decompose(x, out=c, ws=wd)
        bank.reconstruct(c, out=y, ws=wr)
    t = _time(step)
    s = 2 if dtype == torch.bfloat16 else 4
    peak, src = _peak()
    gbs = alg_bytes(B, K, N, M, s) / t / 1e9
    return {"rows": N, "cols": M, "filters": K, "batch": B,
            "coeff_dtype": "bf16" if s == 2 else "f32", "ms": t * 1e3,
            "coeffs_per_s": B * K * N * M / t, "alg_gbs": gbs, "frac_of_hbm_peak": gbs / peak,
            "peak_source": src, "pr_rel_err": float(((y - x).abs().max() / x.abs().max()).item())}


def general_point(bank, B, label, seed=5000):
    """transform_point on a general-kernel bank, plus the device time of
    each launch name in one decomposition + reconstruction pass."""
    from .shearlet import shl_profile_enable, shl_profile_read
    out = dict(transform_point(bank, B, torch.float32, seed), config=label, general=bank.general)
    x = torch.from_numpy(np.stack([synth.cartoon(bank.rows, bank.cols, seed + b)
                                   for b in range(B)]).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    shl_profile_read()
    shl_profile_enable(1)
    bank.reconstruct(bank.decompose(x))
    torch.cuda.synchronize()
    shl_profile_enable(0)
    out["launch_ms"] = {k: round(v["ms"], 4) for k, v in shl_profile_read().items()}
    return out


def general_points():
    pts = []
    for (N, M) in ((480, 640), (500, 500), (509, 509)):
        b = Bank.create(N, M, 4, device=0)
        pts.append(general_point(b, 16, "%dx%d, K=49, B=16" % (N, M)))
        b.close()
    ref = Bank.create(512, 512, 4, device=0)
    info = ref.info()
    g = Bank.from_complex_spectra(info["spectra"], info["idx"], device=0)
    pts.append(general_point(g, 16, "512x512 on the general kernels, K=49, B=16"))
    pts.append(general_point(ref, 16, "512x512 on the half-spectrum kernels, K=49, B=16"))
    return pts


def ray_point(N, A, B):
    """Forward and adjoint ray transform of B phantoms (CUDA-event timing),
    as samples (rays x samples per ray) per second."""
    from .ray import RayTransform
    op = RayTransform(N, A, device=0)
    x = torch.from_numpy(np.stack([synth.ellipse_phantom(synth.random_ellipses(s), N)
                                   for s in range(B)]).astype(np.float32)).cuda()
    p = op.forward(x)
    y = torch.empty_like(x)
    tf = _time(lambda: op.forward(x, out=p))
    ta = _time(lambda: op.adjoint(p, out=y))
    samples = B * A * op.n_det * N
    return {"size": N, "angles": A, "bins": op.n_det, "batch": B, "forward_ms": tf * 1e3,
            "adjoint_ms": ta * 1e3, "forward_samples_per_s": samples / tf,
            "adjoint_samples_per_s": samples / ta}


def small_case(N, B, bf16=False):
    bank = Bank.create(N, N, 4, device=0)
    x = torch.from_numpy(np.stack([synth.cartoon(N, N, s) for s in range(B)]).astype(np.float32)).cuda()
    dt = torch.bfloat16 if bf16 else torch.float32
    for _ in range(2):
        c = bank.decompose(x, dtype=dt)
        r = bank.reconstruct(c)
    torch.cuda.synchronize()
    err = (r - x).abs().max().item()
    print("case %dx%d B=%d K=%d %s: max |rec - x| = %.3g" % (N, N, B, bank.K, dt, err))
    if not err <= (1e-2 if bf16 else 1e-5) * x.abs().max().item():
        raise SystemExit("perfect reconstruction failed")


def bank_point(N, J, reps=3):
    """Wall time of the filter-bank construction: host float64 builder +
    upload (shl_bank_create) against the GPU builder (shl_bank_create_gpu)."""
    import time
    out = {"rows": N, "cols": N, "scales": J}
    for name, gpu in (("host_s", False), ("gpu_s", True)):
        Bank.create(N, N, J, device=0, on_gpu=gpu).close()          # warm-up
        best = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b = Bank.create(N, N, J, device=0, on_gpu=gpu)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
            b.close()
        out[name] = best
    out["filters"] = Bank.create(N, N, J, device=0, on_gpu=True).K
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--case", type=int, nargs=2, metavar=("N", "B"), default=None)
    ap.add_argument("--bf16", action="store_true", help="--case with bfloat16 coefficients")
    ap.add_argument("--general", action="store_true")
    ap.add_argument("--ray", action="store_true")
    args = ap.parse_args()
    from . import _build
    _build.build()
    if args.case:
        small_case(*args.case, bf16=args.bf16)
        return
    if args.ray:
        pts = [ray_point(128, 30, 32), ray_point(512, 180, 8), ray_point(1024, 360, 1)]
        print(json.dumps(pts, indent=1))
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(pts, fh, indent=1)
        return
    if args.general:
        pts = general_points()
        print(json.dumps(pts, indent=1))
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(pts, fh, indent=1)
        return
    res = {"transform": [], "denoise": None, "layer": None, "bank": [], "inpainting": [],
           "general": general_points(),
           "ray": [ray_point(128, 30, 32), ray_point(512, 180, 8), ray_point(1024, 360, 1)]}
    for N, J in ((256, 2), (512, 4), (1024, 4)):
        res["bank"].append(bank_point(N, J))
    b256_2 = Bank.create(256, 256, 2, device=0)
    res["transform"].append(dict(transform_point(b256_2, 1, torch.float32), config="plain 256, K=17"))
    b512 = Bank.create(512, 512, 4, device=0)
    for dt in (torch.float32, torch.bfloat16):
        res["transform"].append(dict(transform_point(b512, 16, dt), config="512, K=49, B=16"))
    b1024 = Bank.create(1024, 1024, 4, device=0)
    for B in (1, 2, 4, 8):
        for dt in (torch.float32, torch.bfloat16):
            res["transform"].append(dict(transform_point(b1024, B, dt), config="1024 sweep"))
    # denoising, 16 x 512, sigma 30/255, threshold 3 sigma RMS_i
    sigma = 30 / 255
    clean, noisy = synth.denoise_batch(16, 512, sigma, seed0=100)
    xn = torch.from_numpy(noisy.astype(np.float32)).cuda()
    ct = torch.from_numpy(clean.astype(np.float32)).cuda()
    t = _time(lambda: apps.denoise(b512, xn, sigma, 3.0))
    den = apps.denoise(b512, xn, sigma, 3.0)
    res["denoise"] = {"batch": 16, "size": 512, "filters": 49, "ms": t * 1e3,
                      "psnr_noisy": apps.psnr(xn, ct).mean().item(),
                      "psnr_denoised": apps.psnr(den, ct).mean().item()}
    # inpainting as in the paper's experiments: 512 x 512, 50 iterations of
    # the hard-threshold iteration, random and squared masks (8 images each)
    for kind in ("random", "squared"):
        clean8, mask8, masked8 = synth.inpaint_batch(8, 512, 0.5, seed0=2000, kind=kind)
        fm = torch.from_numpy(masked8.astype(np.float32)).cuda()
        mk = torch.from_numpy(mask8.astype(np.float32)).cuda()
        c8 = torch.from_numpy(clean8.astype(np.float32)).cuda()
        t = _time(lambda: apps.iht_inpaint(b512, fm, mk, 50), reps=3)
        out = apps.iht_inpaint(b512, fm, mk, 50)
        res["inpainting"].append({"mask": kind, "batch": 8, "size": 512, "filters": 49,
                                  "iterations": 50, "ms": t * 1e3,
                                  "psnr_masked": apps.psnr(fm, c8).mean().item(),
                                  "psnr_inpainted": apps.psnr(out, c8).mean().item()})
    # differentiable layer, 32 x 256, 33 filters, bfloat16 coefficients
    b256_3 = Bank.create(256, 256, 3, device=0)
    c32, n32 = synth.denoise_batch(32, 256, sigma, seed0=1000)
    xl = torch.from_numpy(n32.astype(np.float32)).cuda().requires_grad_(True)

    def layer():
        y = shearlet_rec(shearlet_dec(xl, b256_3, torch.bfloat16), b256_3)
        y.backward(torch.ones_like(y))
    t = _time(layer)
    res["layer"] = {"batch": 32, "size": 256, "filters": 33, "coeff_dtype": "bf16",
                    "ms_fwd_bwd": t * 1e3}
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
