#!/usr/bin/env python
"""Throughput of the wavelet multilevel l1-deblurring V-cycle on one B300.

Workload (one "step" = one complete V-cycle solve, Alg. 4, of one image):
m = 512 synthetic piecewise-constant phantoms (40 rectangles, 20 disks,
intensities U[0,1]), Gaussian PSF sigma = 3 on 15 x 15, 1 % and 5 % noise,
3-level cycles; step s runs combination s mod 12 of {IRLS, MM, SB} x
{Haar, Db4} x {X, D} on image seed s mod 4 with noise 1 % (even blocks of 12
steps) or 5 % (odd blocks). FP32 storage, FP64 reductions.

Metric: deblurred Mpixel/s (whole job, all ranks). Inputs are resident in
HBM when the timed region starts; L2 is flushed (256 MB write) before every
step, outside the CUDA-event pair that times it. `e2e` repeats steps through
the host-buffer C-ABI call (pinned host input, host->device and
device->host copies inside the timed region).

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (see cpu_baseline_sample()).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = 512
SIGMA, PSF_SIZE = 3.0, 15
LEVELS = 3
COMBOS = [(s, w, t) for s in ("irls", "mm", "sb") for w in ("haar", "db4") for t in ("X", "D")]
NOISES = (0.01, 0.05)
L2_FLUSH_BYTES = 256 << 20
# LSQR algorithmic traffic per pixel per iteration, FP32 storage (4-byte words):
# pass F reads v, u_A, u_Lx, u_Ly, w, delta and writes u_A, u_Lx, u_Ly, w, delta
# (11 words); pass B reads u_A, u_Lx, u_Ly, v and writes v (5 words); IRLS
# also reads the two weight planes in both passes (+4 words).
BYTES_PER_PIX_ITER = {"other": 16 * 4, "irls": 20 * 4}
# Measured DRAM bytes per k_lsqr launch on this workload: one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, cold cache) of the timed
# solve's first 80 LSQR launches, on the 128 x 128 and 256 x 256 levels. A
# launch reads its level's vectors once from HBM (19-25 B per pixel) and
# iterates from L2. To be retaken whenever k_lsqr changes.
LSQR_DRAM_BYTES_PER_LAUNCH = 716470
LSQR_DRAM_SCOPE = "ncu, cold cache, mean over the timed solve's first 80 k_lsqr launches (128x128 and 256x256 levels)"


def workload_desc():
    return {"workload": "m512_gauss_s3_15x15_3level_12combos", "m": M, "psf": f"gaussian sigma={SIGMA} {PSF_SIZE}x{PSF_SIZE}",
            "levels": LEVELS, "combos": "irls/mm/sb x haar/db4 x X/D", "noise": "1%,5%",
            "phantom": "40 rect + 20 disk", "precision": "fp32 storage, fp64 reductions",
            "l2": "flushed (256 MB write) before every step"}


def step_spec(s):
    solver, wavelet, transfer = COMBOS[s % len(COMBOS)]
    noise = NOISES[(s // len(COMBOS)) % 2]
    seed = s % 4
    return solver, wavelet, transfer, noise, seed


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ inputs
def make_inputs(api, torch, s, psf_dev):
    """Phantom, PSF and noise from the input generator; b_true = A x_true by
    the library's own forward blur (level 0, FP64)."""
    from paper_2608_17123_b300 import inputs as I
    solver, wavelet, transfer, noise, seed = step_spec(s)
    x_true = I.phantom(M, 40, 20, seed)
    xd = torch.from_numpy(I.to_colmajor(x_true).ravel()).cuda()
    bd = torch.empty_like(xd)
    api.apply_blur(I.gaussian_psf(SIGMA, PSF_SIZE), M, xd, bd)
    b_true = I.from_colmajor(bd.cpu().numpy(), M)
    b = I.add_noise(b_true, I.noise_direction(M, 10_000 + seed), noise)
    return b, x_true


# ------------------------------------------------------------------ sharding
def shard_steps(rank, warmup, steps):
    """Step indices of one rank: every rank solves its own images (weak
    scaling, no data-path collective), rank r taking a disjoint block."""
    total = warmup + steps
    return [rank * total + i for i in range(total)]


def max_over_ranks(t_ms, world):
    """Largest per-rank time (the job's wall time); a collective only when
    there is more than one rank (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(t_ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch
    from paper_2608_17123_b300 import api
    from paper_2608_17123_b300 import inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    ctx = api.Context(torch.cuda.current_device())
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    psf = I.gaussian_psf(SIGMA, PSF_SIZE)
    psf_dev = torch.from_numpy(I.to_colmajor(psf).ravel()).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    total = args.warmup + args.steps
    steps = shard_steps(rank, args.warmup, args.steps)
    # inputs resident in HBM before timing
    dev_inputs = []
    host_inputs = []
    for s in steps:
        b, _ = make_inputs(api, torch, s, psf_dev)
        bb = torch.from_numpy(I.to_colmajor(b).ravel()).cuda()
        dev_inputs.append(bb)
        host_inputs.append(I.to_colmajor(b).ravel())
    x_dev = torch.empty(M * M, dtype=torch.float64, device="cuda")
    per_level_counts = []

    def solve_dev(i):
        solver, wavelet, transfer, _, _ = step_spec(steps[i])
        return api.deblur_solve_device(dev_inputs[i], psf_dev, M, PSF_SIZE, x_dev, solver, wavelet, LEVELS, transfer,
                                       precision="fp32", ctx=ctx, stream=stream.cuda_stream)

    for i in range(args.warmup):
        solve_dev(i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times = []
    for i in range(args.warmup, total):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select exactly the timed steps
        r = solve_dev(i)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        per_level_counts.append((step_spec(steps[i])[0], r["iters"], r["inner"]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = ctx.stats()
    t_total_ms = max_over_ranks(sum(times), world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    pixels = M * M * args.steps * world
    value = pixels / (t_total_ms / 1e3) / 1e6

    # e2e through the host-buffer call (pinned input; copies inside the timed region)
    # --e2e-steps 0 skips this pass (profiling runs only; the line then has no e2e number)
    e2e_steps = max(0, min(args.steps, args.e2e_steps))
    pinned_b = [torch.from_numpy(host_inputs[args.warmup + i]).pin_memory() for i in range(e2e_steps)]
    psf_host = torch.from_numpy(I.to_colmajor(psf).ravel()).pin_memory()
    x_host = torch.empty(M * M, dtype=torch.float64).pin_memory()
    import ctypes as C
    from paper_2608_17123_b300 import _lib as L
    e2e_ms = 0.0
    for i in range(e2e_steps):
        solver, wavelet, transfer, _, _ = step_spec(steps[args.warmup + i])
        o, g = api.make_opts("fp32")
        mu = np.zeros(LEVELS)
        it = np.zeros(LEVELS, dtype=np.int32)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = L.lib().deblur_solve(ctx.handle, C.c_void_p(pinned_b[i].data_ptr()), M, C.c_void_p(psf_host.data_ptr()),
                                  PSF_SIZE, L.SOLVERS[solver], L.WAVELETS[wavelet], LEVELS, L.TRANSFERS[transfer],
                                  C.byref(g), C.byref(o), C.c_void_p(x_host.data_ptr()), mu.ctypes.data,
                                  it.ctypes.data, None, 0, C.c_void_p(stream.cuda_stream))
        L.check(st, ctx.handle)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_value = M * M * e2e_steps * world / (e2e_ms / 1e3) / 1e6 if e2e_steps else None

    # batched and served forms on the same timed images (host buffers, like e2e)
    forms = {}
    if world == 1 and args.forms:
        forms = run_forms(api, ctx, torch, [host_inputs[args.warmup + i] for i in range(args.steps)],
                          [steps[args.warmup + i] for i in range(args.steps)], psf)

    # roofline of the dominant kernel (LSQR persistent kernel)
    peak, peak_kind = load_peaks()
    bytes_alg = (stats["lsqr_pixel_iters_irls"] * BYTES_PER_PIX_ITER["irls"]
                 + stats["lsqr_pixel_iters_other"] * BYTES_PER_PIX_ITER["other"])
    launches = max(1, stats["lsqr_launches"])
    achieved = (bytes_alg / launches) / ((stats["lsqr_ms"] / launches) / 1e3) / 1e9 if stats["lsqr_ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": LSQR_DRAM_BYTES_PER_LAUNCH,
                "traffic_scope": LSQR_DRAM_SCOPE,
                "algorithmic_bytes_per_launch": round(bytes_alg / launches),
                "kernel": "k_lsqr (persistent cooperative LSQR)", "peak_kind": peak_kind,
                "lsqr_share_of_step": round(stats["lsqr_ms"] / t_total_ms, 4) if t_total_ms else None}

    line = {
        "metric": "deblurred Mpixel/s", "value": round(value, 4), "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic phantoms (inputs module), b = A x_true by the library's blur + seeded noise",
        "config": workload_desc(),
        "images_per_s": round(args.steps * world / (t_total_ms / 1e3), 4),
        "e2e": None if e2e_value is None else
               {"value": round(e2e_value, 4), "unit": "Mpixel/s", "steps": e2e_steps,
                "h2d_bytes_per_step": M * M * 8 + PSF_SIZE * PSF_SIZE * 8, "d2h_bytes_per_step": M * M * 8 + LEVELS * 12},
        "gpu_launches": int(stats["kernel_launches"]),
        "roofline": roofline,
        "clocks": clk,
        "counts": {"lsqr_launches": int(stats["lsqr_launches"]), "gcv_calls": int(stats["gcv_calls"]),
                   "outer_iterations": int(stats["outer_iterations"])},
        "step_split": {"lsqr_ms_per_step": round(stats["lsqr_ms"] / args.steps, 2),
                       "gcv_ms_per_step": round(stats.get("gcv_ms", 0.0) / args.steps, 2)},
    }
    line.update(forms)
    return line, per_level_counts, times


def run_forms(api, ctx, torch, bs, step_ids, psf):
    """Images/s of the plain one-at-a-time host call, the batched call
    (deblur_solve_batch) and the serving loop (db_server_*, all requests
    queued at once) on the same images, with the largest relative difference
    of the batched and served reconstructions from the plain ones; then a
    Poisson request stream at 80 % of the batched throughput (each image
    twice) with its p50/p99 latency."""
    from paper_2608_17123_b300 import inputs as I
    imgs = [I.from_colmajor(b, M) for b in bs]
    specs = [step_spec(s) for s in step_ids]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [api.deblur_solve(b, psf, sp[0], sp[1], LEVELS, sp[2], precision="fp32", ctx=ctx)
             for b, sp in zip(imgs, specs)]
    t_plain = time.perf_counter() - t0
    probs = [dict(b=b, psf=psf, solver=sp[0], wavelet=sp[1], levels=LEVELS, transfer=sp[2])
             for b, sp in zip(imgs, specs)]
    t0 = time.perf_counter()
    batched = api.deblur_solve_batch(probs, precision="fp32", ctx=ctx)
    t_batch = time.perf_counter() - t0
    srv = api.Server(max_resident=len(imgs), max_m=M)
    t0 = time.perf_counter()
    tickets = [srv.submit(b, psf, sp[0], sp[1], LEVELS, sp[2]) for b, sp in zip(imgs, specs)]
    served, lat = [], []
    for tk in tickets:
        r, l = srv.poll(tk)
        served.append(r)
        lat.append(l)
    t_srv = time.perf_counter() - t0
    srv.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    # Poisson arrivals at 80 % of the batched throughput, each image twice:
    # latency from submit to completion as the server reports it
    rng = np.random.default_rng(2026)
    rate = 0.8 * len(imgs) / t_batch
    order = [i % len(imgs) for i in range(2 * len(imgs))]
    gaps = rng.exponential(1.0 / rate, size=len(order))
    srv = api.Server(max_resident=len(imgs), max_m=M)
    t0 = time.perf_counter()
    tks, t_next = [], 0.0
    for k, i in enumerate(order):
        t_next += gaps[k]
        while time.perf_counter() - t0 < t_next:
            time.sleep(0.0005)
        sp = specs[i]
        tks.append(srv.submit(imgs[i], psf, sp[0], sp[1], LEVELS, sp[2]))
    lat_p = [srv.poll(tk)[1] for tk in tks]
    t_poisson = time.perf_counter() - t0
    srv.close()
    n = len(imgs)
    lat_sorted = sorted(lat)
    poisson = {"rate_per_s": round(rate, 3), "requests": len(order), "images_per_s": round(len(order) / t_poisson, 4),
               "p50_ms": round(float(np.percentile(lat_p, 50)), 2), "p99_ms": round(float(np.percentile(lat_p, 99)), 2)}
    return {
        "plain_images_per_s": round(n / t_plain, 4),
        "batched": {"images_per_s": round(n / t_batch, 4), "images": n, "call": "deblur_solve_batch",
                    "max_rel_diff_vs_plain": max(rel(b["x"], p["x"]) for b, p in zip(batched, plain))},
        "serving": {"images_per_s": round(n / t_srv, 4), "requests": n, "arrival": "all queued at t=0",
                    "p50_ms": round(float(np.percentile(lat_sorted, 50)), 2),
                    "p99_ms": round(float(np.percentile(lat_sorted, 99)), 2),
                    "max_rel_diff_vs_plain": max(rel(q["x"], p["x"]) for q, p in zip(served, plain)),
                    "poisson": poisson},
    }


# ------------------------------------------------------------------ oracle sample
def gcv_calls(solver, level, outer):
    """GCV estimates a level makes (the schedule of Sec. 3 as implemented)."""
    if solver == "irls":
        if level == 0 and LEVELS >= 3:
            return 1 + (1 if outer > 3 else 0)
        return outer
    return min(3, outer)


def cpu_baseline_sample(counts, budget_s=20.0):
    """Time the FP64 oracle on a bounded sample of the workload and scale it
    to Mpixel/s: per level, oracle LSQR iterations on that level's problem
    (m = 512, 256, 128; MM form, Db4 hierarchy) and one oracle GCV (projected,
    k = 40) on the 128 x 128 level, scaled by pixel count to the other levels;
    the per-solve work (LSQR iterations and GCV calls per level) comes from
    `counts` (the GPU run's own counts for the same steps) or, without them,
    from the work model below."""
    try:
        from threadpoolctl import threadpool_limits
        limiter, cores = threadpool_limits(limits=1), 1
    except ImportError:           # not installed: BLAS keeps its own threads
        import contextlib
        limiter, cores = contextlib.nullcontext(), os.cpu_count()
    from oracle import operators as O
    from oracle import solvers as S
    from paper_2608_17123_b300 import inputs as I
    with limiter:
        g = I.gaussian_factor(SIGMA, PSF_SIZE)
        A = O.KronOp.from_factors(M, g, g)
        x_true = I.phantom(M, 40, 20, 0)
        b = I.add_noise(A.apply(x_true), I.noise_direction(M, 10_000), 0.01)
        As, bs = [A], [b]
        for _ in range(LEVELS - 1):
            As.append(As[-1].coarsen("db4"))
            bs.append(O.restrict(bs[-1], "db4"))
        t_iter = []
        t0_all = time.perf_counter()
        for lvl in range(LEVELS):
            mm = As[lvl].m
            z = (np.zeros((mm - 1, mm)), np.zeros((mm, mm - 1)))
            sub = S.Subproblem(As[lvl], bs[lvl], c=z)
            its = 12 if lvl == 0 else 20
            t = time.perf_counter()
            _, k = sub.solve(1e-3, np.zeros((mm, mm)), S.opts_with(lsqr_maxit=its, lsqr_atol=0, lsqr_btol=0))
            t_iter.append((time.perf_counter() - t) / max(k, 1))
        sub = S.Subproblem(As[-1], bs[-1], c=None)
        t = time.perf_counter()
        sub.gcv(S.opts_with(proj_dim=40, proj_dim_max=40))
        t_gcv_c = time.perf_counter() - t
        elapsed = time.perf_counter() - t0_all
    t_gcv = [t_gcv_c * (4 ** (LEVELS - 1 - l)) for l in range(LEVELS)]
    tot_t, tot_pix = 0.0, 0
    for solver, iters, inner in counts:
        for l in range(LEVELS):
            tot_t += inner[l] * t_iter[l] + gcv_calls(solver, l, iters[l]) * t_gcv[l]
        tot_pix += M * M
    value = tot_pix / tot_t / 1e6
    sample = (f"oracle LSQR iterations on the m=512/256/128 levels ({t_iter[0]*1e3:.1f}/{t_iter[1]*1e3:.1f}/"
              f"{t_iter[2]*1e3:.1f} ms per iteration) and one projected GCV (k=40) on the 128x128 level "
              f"({t_gcv_c:.2f} s, scaled by pixel count), combined with the per-level LSQR iteration and GCV "
              f"counts of {len(counts)} solves; {elapsed:.1f} s of CPU work")
    return {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": sample}


# Per-solve work model (LSQR iterations and outer iterations per level, finest
# first) of the 12 combinations on this workload, from a B300 run of this
# benchmark; used by the reference arm, which has no GPU run to count from.
WORK_MODEL = [
    ("irls", [18, 50, 50], [1366, 3916, 2124]),
    ("mm", [19, 50, 50], [1343, 2607, 727]),
    ("sb", [31, 50, 50], [685, 2761, 999]),
]


def run_reference(args, rank, world):
    if rank != 0:
        return None
    samples = []
    for _ in range(args.warmup + args.steps):
        t = time.perf_counter()
        cb = cpu_baseline_sample(WORK_MODEL, budget_s=5.0)
        samples.append((cb, time.perf_counter() - t))
    timed = samples[args.warmup:]
    value = statistics.mean(c["value"] for c, _ in timed)
    cb = dict(timed[-1][0])
    cb["value"] = value
    line = {"metric": "deblurred Mpixel/s", "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * M * M / (value * 1e6), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_desc(), "impl": "reference",
            "cpu_baseline": cb, "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the batched / serving comparison")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    line, counts, _ = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample(counts)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
