#!/usr/bin/env python3
"""Throughput of the shearlet transform hot path on GB300.

One step = shearlet decomposition + reconstruction (fwd + inv) of a batch of
B = 16 images of 512 x 512 with the K = 49 filters of 4 scales (shear levels
1, 1, 2, 2), float32 coefficients.  Metric: shearlet coefficients per second,
B K N^2 / t(step).  Inputs are seeded synthetic cartoons (the paper's images
are not available).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank processes its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_IMG, K_FILT, B_IMG, SCALES = 512, 49, 16, 4
METRIC = "Shearlet coeffs/s fwd+inv at 512^2, 49 filters"
UNIT = "coeffs/s"
L2_FLUSH_BYTES = 512 << 20
SWEEP_STEPS = 20                 # timed steps per point of the 1024 x 1024 sweep


def _config(extra=None):
    cfg = {"workload": "decompose+reconstruct, B=16 x 512x512 float32 images, K=49 "
                       "(4 scales, shear levels 1,1,2,2), float32 coefficients",
           "rows": N_IMG, "cols": N_IMG, "filters": K_FILT, "global_batch": B_IMG,
           "coeff_dtype": "f32", "l2": "flushed between timed steps (512 MiB write); "
                                        "coefficients (822 MB) also exceed L2"}
    if extra:
        cfg.update(extra)
    return cfg


def _algorithmic_bytes(B, K, N, M, s=4):
    """Step bytes: dec reads images + filters, writes coefficients; rec reads
    coefficients + filters + 1/W, writes images (half-spectrum float32 filters)."""
    H = N * (M // 2 + 1)
    dec = B * (4 * N * M + s * K * N * M) + 4 * K * H
    rec = B * (s * K * N * M + 4 * N * M) + 4 * K * H + 4 * H
    return dec, rec


# ------------------------------------------------- ncu traffic (profiles/)
KERNEL_SOURCES = ("fast.cu", "warp_fft.cuh", "fft_core.cuh", "internal.h")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the transform kernels' sources;
    the ncu summaries record it so that a stale figure is not reported."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_04591_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel):
    """DRAM bytes per subband of ``kernel`` from the committed ncu summary
    profiles/<kernel>_512_k49.md, or None if it is absent or was taken on
    other kernel sources."""
    path = os.path.join(ROOT, "profiles", "%s_512_k49.md" % kernel)
    try:
        lines = open(path).read().splitlines()
        cur = kernel_source_hash()
    except OSError:
        return None
    vals = {}
    for line in lines:
        key, sep, val = line.partition(":")
        if sep:
            vals[key.strip()] = val.strip()
    if vals.get("source_sha256_16") != cur:
        return None
    try:
        return float(vals["traffic_bytes_per_subband"])
    except (KeyError, ValueError):
        return None


def _e2e_block(units_per_step, io_bytes, variants):
    """The end-to-end figure: the fastest of the measured ways of running a
    step from pinned host images to pinned host results through the public
    API (each step copies or reads its inputs and results over the
    CPU-GPU link inside the timed region), with every variant listed."""
    best = min(variants, key=lambda v: v[0])
    return {"value": units_per_step / best[0], "unit": UNIT,
            "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
            "transfer": best[1], "max_rel_err": best[2],
            "variants": [{"value": units_per_step / t, "unit": UNIT, "ms_per_step": t * 1e3,
                          "transfer": d} for t, d, _ in variants]}


def kernel_alg_bytes(name, B, K, N, M, s=4):
    """Algorithmic HBM bytes one step's launches of kernel `name` move
    (images, coefficients, filter and 1/W half spectra; no intermediates)."""
    H = N * (M // 2 + 1)
    img, coef, filt = B * N * M * 4, B * K * N * M * s, K * H * 4
    return {
        "rows_r2c_image": img, "rows_c2r_image": img, "lines_fwd_image": 0,
        "dec_lines": filt, "dec_lines_tc": filt, "rec_lines": filt + H * 4,
        "rows_c2r_coeffs": coef, "rows_r2c_coeffs": coef,
        "pair_dec": coef + filt, "pair_rec": coef + filt, "pair_final": H * 4,
        "dec_pipe": coef + filt, "rows_shrink": 0,
    }.get(name, 0)


def roofline(prof, steps, B, K, N, M, s, peak, peak_src):
    """Roofline of the kernel with the most device time in `prof` (the
    library's per-launch CUDA-event profile over `steps` steps)."""
    if not prof:
        return None
    name, rec = max(prof.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = rec["ms"] / rec["launches"]
    per_step_launches = rec["launches"] / steps
    alg = kernel_alg_bytes(name, B, K, N, M, s) / per_step_launches
    achieved = alg / (per_launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src, "launch_ms": per_launch_ms,
            "algorithmic_bytes_per_launch": alg, "launches_per_step": per_step_launches}


# ------------------------------------------------------- multi-rank logic
def rank_seeds(rank: int, batch: int, base: int = 100):
    """Image seeds of one replica: each rank decomposes its own batch."""
    return [base + rank * batch + b for b in range(batch)]


def reduce_max_time(t_local: float, dist, device) -> float:
    """Max over ranks of a step time (the slowest replica bounds the job)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, t_step: float) -> float:
    """Whole-job throughput: units processed by all ranks / max step time."""
    return units_per_rank * world / t_step


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device_index=0):
        self.samples = []
        self.proc = None
        self.dev = device_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------------- CPU
_ORACLE_BANK = []


def _oracle_sample(seconds_target=12.0, max_images=B_IMG, first_seed=100):
    """Oracle dec+rec on whole images of the workload until ~seconds_target."""
    import numpy as np
    from oracle import bank as Bk
    from oracle import transform as OT
    from paper_2006_04591_gb300 import synth
    if not _ORACLE_BANK:
        _ORACLE_BANK.append(Bk.shearlet_bank(N_IMG, N_IMG, SCALES))
    ref = _ORACLE_BANK[0]
    done, t0 = 0, time.perf_counter()
    while done < max_images:
        x = synth.cartoon(N_IMG, N_IMG, first_seed + done).astype(np.float32)
        c = OT.decompose(x, ref["psi_hat"]).real
        OT.reconstruct(c, ref["psi_hat"])
        done += 1
        if time.perf_counter() - t0 >= seconds_target:
            break
    dt = time.perf_counter() - t0
    return done, dt


# ------------------------------------------------- CPU table (oracle only)
_TABLE_BANK = {}


def _table_init(n, J):
    from oracle import bank as Bk
    _TABLE_BANK["ref"] = Bk.shearlet_bank(n, n, J)


def _table_work(args):
    """dec + rec of one seeded cartoon with the worker's oracle bank."""
    import numpy as np
    from oracle import transform as OT
    from paper_2006_04591_gb300 import synth
    n, seed = args
    ref = _TABLE_BANK["ref"]
    x = synth.cartoon(n, n, seed).astype(np.float32)
    c = OT.decompose(x, ref["psi_hat"]).real
    OT.reconstruct(c, ref["psi_hat"])
    return 0


def run_cpu_table():
    """The FP64 oracle (numpy float64, single-threaded FFTs) on the host cores
    for the plain-transform, metric and 1024 x 1024 workloads: one process,
    and a spawn process pool over the images (bank built in each worker
    before the timed pass).  Prints one JSON line."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    rows = []
    for n, J, B in ((256, 2, 1), (512, 4, 16), (1024, 4, 1), (1024, 4, 8)):
        _table_init(n, J)
        seeds = [(n, 100 + b) for b in range(B)]
        t0 = time.perf_counter()
        for a in seeds:
            _table_work(a)
        t1 = time.perf_counter() - t0
        row = {"rows": n, "scales": J, "batch": B, "one_process_s": t1}
        if B > 1:
            nw = min(cores, B)
            with ctx.Pool(nw, initializer=_table_init, initargs=(n, J)) as pool:
                pool.map(_table_work, seeds, chunksize=1)          # workers up, banks built
                t0 = time.perf_counter()
                pool.map(_table_work, seeds, chunksize=1)
                row["all_cores_s"] = time.perf_counter() - t0
                row["processes"] = nw
        rows.append(row)
    print(json.dumps({"cpu_table": rows, "cores": cores, "kind": "oracle (numpy float64)"}))
    return 0


def _cpu_cores_used():
    # numpy.fft (pocketfft) runs on one thread; the oracle loops in Python.
    return 1


def run_reference(args):
    """The FP64 oracle on the host: each step decomposes and reconstructs one
    image of the workload (a bounded sample of the 16-image batch), and the
    line reports exactly that: ms_per_step is the time of one such step and
    value = K N^2 / that time, in the GPU arm's metric, unit and config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = []
    for s in range(args.warmup + args.steps):
        n, dt = _oracle_sample(seconds_target=4.0, max_images=1, first_seed=100 + s % B_IMG)
        if s >= args.warmup:
            per_step.append(dt / n)
    t_step = statistics.mean(per_step)
    value = K_FILT * N_IMG * N_IMG / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config({"parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1
                                          else "single"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cpu_cores_used(),
                         "kind": "oracle",
                         "sample": "one of the 16 images per step (dec+rec, K=49, 512^2, "
                                   "FP64 numpy oracle); %d timed steps" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------- GPU
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2006_04591_gb300 import shearlet as S
    from paper_2006_04591_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2006_04591_gb300 import _build
    _build.build()
    bank = S.Bank.create(N_IMG, N_IMG, SCALES, device=local)
    assert bank.K == K_FILT
    B, N, K = B_IMG, N_IMG, K_FILT
    x_host = np.stack([synth.cartoon(N, N, sd) for sd in rank_seeds(rank, B)]).astype(np.float32)
    x = torch.from_numpy(x_host).to(dev)
    coeffs = torch.empty((B, K, N, N), dtype=torch.float32, device=dev)
    xr = torch.empty((B, N, N), dtype=torch.float32, device=dev)
    ws_d = bank.workspace(S.SHL_OP_DECOMPOSE, B)
    ws_r = bank.workspace(S.SHL_OP_RECONSTRUCT, B)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        bank.decompose(x, out=coeffs, ws=ws_d)
        bank.reconstruct(coeffs, out=xr, ws=ws_r)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    err = ((xr - x).abs().max() / x.abs().max()).item()

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)     # sampled while the GPU runs the timed passes below
    clocks.start()
    n0 = S.shl_launch_count()
    times = timed(step, args.steps)
    launches = S.shl_launch_count() - n0
    t_step = reduce_max_time(sum(times) / len(times) / 1e3, dist if world > 1 else None, dev)
    if world > 1:
        dist.barrier()

    # per-kernel timing with CUDA events on the launch stream (separate pass)
    S.shl_profile_enable(1)
    S.shl_profile_read()
    prof_times = timed(step, args.steps)
    S.shl_profile_enable(0)
    prof = S.shl_profile_read()
    t_prof = sum(prof_times) / len(prof_times) / 1e3

    # end to end through the public API with pinned host buffers: the images
    # go in and come out of host memory every step.  Primary: the library
    # reads the pinned input and writes the pinned output itself over the
    # CPU-GPU link (first and last kernel); also measured: explicit copies
    # into and out of device buffers around the same calls.
    xh = torch.from_numpy(x_host).pin_memory()
    outh = torch.empty((B, N, N), dtype=torch.float32).pin_memory()

    def e2e_step():
        bank.decompose(xh, out=coeffs, ws=ws_d)
        bank.reconstruct(coeffs, out=outh, ws=ws_r)

    def e2e_copy_step():
        xd = xh.to(dev, non_blocking=True)
        bank.decompose(xd, out=coeffs, ws=ws_d)
        bank.reconstruct(coeffs, out=xr, ws=ws_r)
        outh.copy_(xr, non_blocking=True)

    # the same calls pipelined over two streams, one half batch each: one
    # half's host-to-device copy and device-to-host read overlap the other
    # half's transforms
    halves = [(0, B // 2), (B // 2, B)]
    side = [torch.cuda.Stream(dev) for _ in halves]
    ws_h = [(bank.workspace(S.SHL_OP_DECOMPOSE, hb - ha), bank.workspace(S.SHL_OP_RECONSTRUCT, hb - ha))
            for ha, hb in halves]
    xd_h = [torch.empty((hb - ha, N, N), dtype=torch.float32, device=dev) for ha, hb in halves]

    def e2e_pipe_step():
        for (ha, hb), s, (wd, wr), xd in zip(halves, side, ws_h, xd_h):
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                xd.copy_(xh[ha:hb], non_blocking=True)
                bank.decompose(xd, out=coeffs[ha:hb], ws=wd)
                bank.reconstruct(coeffs[ha:hb], out=xr[ha:hb], ws=wr)
                outh[ha:hb].copy_(xr[ha:hb], non_blocking=True)
        for s in side:
            stream.wait_stream(s)

    def e2e_pipe_mapped_step():
        for (ha, hb), s, (wd, wr) in zip(halves, side, ws_h):
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                bank.decompose(xh[ha:hb], out=coeffs[ha:hb], ws=wd)
                bank.reconstruct(coeffs[ha:hb], out=outh[ha:hb], ws=wr)
        for s in side:
            stream.wait_stream(s)

    for _ in range(3):
        e2e_step()
        e2e_copy_step()
        e2e_pipe_step()
        e2e_pipe_mapped_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_times = timed(e2e_step, args.steps)
    t_e2e = reduce_max_time(sum(e2e_times) / len(e2e_times) / 1e3, dist if world > 1 else None, dev)
    e2e_err = float(np.abs(outh.numpy() - x_host).max() / np.abs(x_host).max())
    if world > 1:
        dist.barrier()
    copy_times = timed(e2e_copy_step, args.steps)
    t_copy = reduce_max_time(sum(copy_times) / len(copy_times) / 1e3, dist if world > 1 else None, dev)
    copy_err = float(np.abs(outh.numpy() - x_host).max() / np.abs(x_host).max())
    if world > 1:
        dist.barrier()
    pipe_times = timed(e2e_pipe_step, args.steps)
    t_pipe = reduce_max_time(sum(pipe_times) / len(pipe_times) / 1e3, dist if world > 1 else None, dev)
    pipe_err = float(np.abs(outh.numpy() - x_host).max() / np.abs(x_host).max())
    if world > 1:
        dist.barrier()
    pm_times = timed(e2e_pipe_mapped_step, args.steps)
    t_pm = reduce_max_time(sum(pm_times) / len(pm_times) / 1e3, dist if world > 1 else None, dev)
    pm_err = float(np.abs(outh.numpy() - x_host).max() / np.abs(x_host).max())
    if world > 1:
        dist.barrier()

    # the same step with bfloat16-stored coefficients (RNE), its own roofline
    c16 = torch.empty((B, K, N, N), dtype=torch.bfloat16, device=dev)

    def step16():
        bank.decompose(x, out=c16, ws=ws_d)
        bank.reconstruct(c16, out=xr, ws=ws_r)

    for _ in range(3):
        step16()
    torch.cuda.synchronize()
    err16 = ((xr - x).abs().max() / x.abs().max()).item()
    t16 = reduce_max_time(sum(timed(step16, args.steps)) / args.steps / 1e3,
                          dist if world > 1 else None, dev)
    S.shl_profile_enable(1)
    S.shl_profile_read()
    timed(step16, args.steps)
    S.shl_profile_enable(0)
    prof16 = S.shl_profile_read()
    del c16
    clock_info = clocks.stop()
    clock_info["window"] = "timed, per-kernel-event and end-to-end passes"

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # the 1024 x 1024 workload (K = 49) at batches 1..8, float32 and bfloat16
    # coefficients: decompose + reconstruct per step, CUDA events, the L2
    # flushed between steps
    sweep = []
    if world == 1 and not args.no_sweep:
        n5 = 1024
        b5 = S.Bank.create(n5, n5, SCALES, device=local)
        x5 = torch.from_numpy(np.stack([synth.cartoon(n5, n5, 5000 + i) for i in range(8)])
                              .astype(np.float32)).to(dev)
        for b_ in (1, 2, 4, 8):
            xs, xo = x5[:b_], torch.empty((b_, n5, n5), dtype=torch.float32, device=dev)
            wd = b5.workspace(S.SHL_OP_DECOMPOSE, b_)
            wr = b5.workspace(S.SHL_OP_RECONSTRUCT, b_)
            for dt, s_ in ((torch.float32, 4), (torch.bfloat16, 2)):
                cs = torch.empty((b_, b5.K, n5, n5), dtype=dt, device=dev)

                def step5():
                    b5.decompose(xs, out=cs, ws=wd)
                    b5.reconstruct(cs, out=xo, ws=wr)

                for _ in range(3):
                    step5()
                torch.cuda.synchronize()
                err5 = ((xo - xs).abs().max() / xs.abs().max()).item()
                t5 = sum(timed(step5, SWEEP_STEPS)) / SWEEP_STEPS / 1e3
                d5, r5 = _algorithmic_bytes(b_, b5.K, n5, n5, s=s_)
                sweep.append({"batch": b_, "coeff_dtype": "f32" if s_ == 4 else "bf16 (RNE)",
                              "ms_per_step": t5 * 1e3, "value": b_ * b5.K * n5 * n5 / t5,
                              "unit": UNIT, "frac_of_peak": (d5 + r5) / t5 / 1e9 / hbm_peak,
                              "pr_rel_err": err5})
                del cs
        del x5, b5

    coeffs_per_step = B * K * N * N * world
    value = job_value(B * K * N * N, world, t_step)
    dec_b, rec_b = _algorithmic_bytes(B, K, N, N)

    # dominant kernel and its algorithmic bytes per launch
    roof = roofline(prof, args.steps, B, K, N, N, 4, hbm_peak, peak_src)
    if roof is not None:
        per_sub = _profiled_traffic(roof["kernel"])
        roof["traffic"] = (per_sub * (B * K) / roof["launches_per_step"]
                           if per_sub is not None else None)

    step_alg = dec_b + rec_b
    dec16, rec16 = _algorithmic_bytes(B, K, N, N, s=2)
    bf16_block = {
        "coeff_dtype": "bf16 (RNE)", "ms_per_step": t16 * 1e3,
        "value": job_value(B * K * N * N, world, t16), "unit": UNIT,
        "vs_f32_time": t16 / t_step,
        "step_hbm": {"algorithmic_bytes": dec16 + rec16,
                     "achieved_gbs": (dec16 + rec16) / t16 / 1e9,
                     "frac_of_peak": (dec16 + rec16) / t16 / 1e9 / hbm_peak},
        "roofline": roofline(prof16, args.steps, B, K, N, N, 2, hbm_peak, peak_src),
        "kernels": {k: {"launches_per_step": v["launches"] / args.steps,
                        "ms_per_step": v["ms"] / args.steps} for k, v in prof16.items()},
        "pr_rel_err": err16,
    }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config({"parallelism": "replicas" if world > 1 else "single"}),
        "step_hbm": {"algorithmic_bytes": step_alg,
                     "achieved_gbs": step_alg / t_step / 1e9,
                     "frac_of_peak": step_alg / t_step / 1e9 / hbm_peak,
                     "peak": hbm_peak, "peak_source": peak_src},
        "roofline": roof,
        "kernels": {k: {"launches_per_step": v["launches"] / args.steps,
                        "ms_per_step": v["ms"] / args.steps} for k, v in prof.items()},
        "profiled_ms_per_step": t_prof * 1e3,
        "e2e": _e2e_block(coeffs_per_step, B * N * N * 4, [
            (t_e2e, "pinned host images read and written by the first and last kernels over "
                    "the CPU-GPU link", e2e_err),
            (t_copy, "cudaMemcpyAsync H2D / D2H around the calls", copy_err),
            (t_pipe, "two streams, one half batch each: H2D copy, decompose, reconstruct, D2H "
                     "copy, the halves overlapping", pipe_err),
            (t_pm, "two streams, one half batch each, the kernels reading and writing the "
                   "pinned host images, the halves overlapping", pm_err)]),
        "bf16": bf16_block,
        "sweep_1024": sweep or None,
        "gpu_launches": launches,
        "clocks": clock_info,
        "pr_rel_err": err,
    }
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            n, dt = _oracle_sample(seconds_target=args.cpu_seconds)
            cpu_val = n * K * N * N / dt
            line["cpu_baseline"] = {"value": cpu_val, "unit": UNIT, "cores": _cpu_cores_used(),
                                    "kind": "oracle",
                                    "sample": "%d of the 16 images, dec+rec K=49 at 512^2, "
                                              "FP64 numpy oracle, %.1f s" % (n, dt)}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the 1024 x 1024 batch sweep (sweep_1024)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the FP64 oracle at several workloads on the host cores and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_table:
        return run_cpu_table()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
