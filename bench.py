#!/usr/bin/env python
"""Throughput of the wavelet multilevel l1-deblurring V-cycle on one B300.

Workload: the m = 512 workload -- a 512 x 512 synthetic piecewise-constant
phantom (40 rectangles, 20 disks, intensities U[0,1], seed 0), Gaussian PSF
sigma = 3 on 15 x 15, b = A x_true + noise at 1 % or 5 %, rounded to float32,
deblurred by 3-level V-cycles (Alg. 4) under all 12 combinations of
{IRLS, MM, SB} x {Haar, Db4} x {X, D}. FP32 storage; LSQR norms and Krylov
dot products as double-float sums of exact products; scalar recurrences, GCV
selection and stopping tests in FP64.

One step = one batch: the 24 cases of the workload (the 12 combinations at
both noise levels) in one deblur_solve_batch call on device buffers
(--batch 12: the 12 combinations of one noise level, alternating).
Metric: deblurred Mpixel/s (whole job, all ranks). Inputs are resident in
HBM when the timed region starts; L2 is flushed (256 MB write) before every
step, outside the CUDA-event pair that times it.

Beside it on the same line: `plain` (the same images, one deblur_solve
each), `e2e` (the same batches through the host-buffer call: copies in and
out inside the timed region), `oracle_parity` (every case against the FP64
oracle's stored result, tests/golden/m512_oracle), `serving` (the server
under all-at-once and Poisson arrivals, p50/p99), `large` (m = 2048, BF16,
5-level Db4 solves of the Gaussian 31 x 31 and 21-pixel motion blurs), and
`cpu_baseline`.

Other modes: --workload batch | serve | study (see their functions), and
--impl reference: the FP64 CPU oracle on a bounded sample of the workload
(see run_reference()).
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
SEED = 0
GOLDEN = os.path.join(ROOT, "tests", "golden", "m512_oracle")
L2_FLUSH_BYTES = 256 << 20

# Large-image workload (m = 2048, 5-level Db4, BF16 storage): steps cycle
# through these (PSF, solver, transfer) cases.
LARGE_M = 2048
LARGE_CASES = [("gauss31", "mm", "X"), ("motion21", "irls", "D"), ("gauss31", "sb", "D"),
               ("motion21", "mm", "X"), ("gauss31", "irls", "X"), ("motion21", "sb", "D")]


def lsqr_bytes_per_pixel_iter(elem, x_elem, irls):
    """Algorithmic LSQR traffic per pixel per iteration: pass F reads v,
    u_A, u_Lx, u_Ly, w and delta and writes u_A, u_Lx, u_Ly, w, delta; pass B
    reads u_A, u_Lx, u_Ly, v and writes v -- 14 storage words and 2 words of
    the iterate type (delta); IRLS also reads the two weight planes in both
    passes (+4 storage words)."""
    return 14 * elem + 2 * x_elem + (4 * elem if irls else 0)


# DRAM traffic of k_lsqr from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/k_lsqr_dram_single_launch.md and
# profiles/k_lsqr_dram_bench_step.md), to be retaken whenever k_lsqr
# changes: (kind, value, scope). "per_launch": bytes per launch measured on
# the line's own command; "per_pixel_iteration": bytes per LSQR
# pixel-iteration of a captured launch, times the pixel-iterations of an
# average launch of the line.
LSQR_DRAM = {
    "m512": ("per_launch", 1.2988e9,
             "measured: the 150 k_lsqr launches of one timed step of this command (ncu, dram__bytes_read.sum + "
             "dram__bytes_write.sum, 115.8 + 79.0 GB per step), averaged per launch; 28 % of their algorithmic "
             "bytes, the rest served by L2"),
    "large": ("per_pixel_iteration", 4.45,
              "scaled from three captured BF16 m = 2048 single-level LSQR launches of the direct path "
              "(0.050 GB read + 1.835 GB written per launch of 4.24e8 pixel-iterations = 4.45 B per "
              "pixel-iteration) to the pixel-iterations of an average finest-level launch"),
}


def lsqr_traffic(key, pixel_iters_per_launch):
    kind, val, scope = LSQR_DRAM[key]
    if kind == "per_launch":
        return round(val), scope
    return round(val * pixel_iters_per_launch), scope


def workload_desc(batch=24):
    return {"workload": "m512_gauss_s3_15x15_3level_12combos", "m": M, "psf": f"gaussian sigma={SIGMA} {PSF_SIZE}x{PSF_SIZE}",
            "levels": LEVELS, "combos": "irls/mm/sb x haar/db4 x X/D", "noise": "1%,5%", "seed": SEED,
            "phantom": "40 rect + 20 disk", "precision": "fp32 storage, double-float (compensated fp32) sums, "
            "fp64 scalar recurrences / GCV / stopping tests",
            "step": ("one deblur_solve_batch call: the 12 combinations at one noise level" if batch == 12 else
                     "one deblur_solve_batch call: all 24 cases (12 combinations x 2 noise levels)"),
            "l2": "flushed (256 MB write) before every step"}


def step_spec(s):
    solver, wavelet, transfer = COMBOS[s % len(COMBOS)]
    noise = NOISES[(s // len(COMBOS)) % 2]
    return solver, wavelet, transfer, noise


def case_name(solver, wavelet, transfer, noise):
    return f"{solver}-{wavelet}-{transfer}-{noise:g}"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def load_golden():
    p = os.path.join(GOLDEN, "index.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


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
def make_b(api, torch, m, x_true, psf, noise, noise_seed):
    """b = A x_true + noise, with A x_true by the library's own level-0 blur
    (FP64), rounded to float32 (the values the FP32 path stores)."""
    from paper_2608_17123_b300 import inputs as I
    xd = torch.from_numpy(I.to_colmajor(x_true).ravel()).cuda()
    bd = torch.empty_like(xd)
    api.apply_blur(psf, m, xd, bd)
    b_true = I.from_colmajor(bd.cpu().numpy(), m)
    b = I.add_noise(b_true, I.noise_direction(m, noise_seed), noise)
    return b.astype(np.float32).astype(np.float64)


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


# ------------------------------------------------------------------ parity
def parity_summary(results, golden):
    """Every timed step against the FP64 oracle's stored result of its case:
    x on the stored pixel sample (relative 2-norm), outer iterations and
    gamma per level."""
    if golden is None:
        return {"available": False, "why": "tests/golden/m512_oracle/index.json missing"}
    idx = np.load(os.path.join(GOLDEN, "sample_index.npy"))
    rows = []
    for (name, x_colmajor, iters, mu) in results:
        c = golden["cases"].get(name)
        if c is None:
            continue
        xo = np.load(os.path.join(GOLDEN, name + ".npz"))["x_samples"].astype(np.float64)
        xs = x_colmajor[idx]
        dx = float(np.linalg.norm(xs - xo) / np.linalg.norm(xo))
        dit = int(max(abs(a - b) for a, b in zip(iters, c["iters"])))
        dmu = float(max(abs(a - b) / b for a, b in zip(mu, c["mu"])))
        rows.append((name, dx, dit, dmu, c["spread_x"], max(c["spread_mu"])))
    if not rows:
        return {"available": False, "why": "no timed step has a stored oracle case"}
    return {"available": True, "reference": "FP64 oracle, tests/golden/m512_oracle (16384-pixel sample)",
            "cases_compared": len(rows),
            "max_rel_diff_x": float(max(r[1] for r in rows)),
            "median_rel_diff_x": float(np.median([r[1] for r in rows])),
            "x_within_1e-4": int(sum(bool(r[1] <= 1e-4) for r in rows)),
            "iters_within_1": int(sum(bool(r[2] <= 1) for r in rows)),
            "mu_within_1pct": int(sum(bool(r[3] <= 1e-2) for r in rows)),
            "max_rel_diff_mu": float(max(r[3] for r in rows)),
            "max_oracle_spread_x": float(max(r[4] for r in rows)),
            "worst_x": sorted(rows, key=lambda r: -r[1])[0][0]}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    """Timed steps: each step deblurs one batch in one deblur_solve_batch call
    on device buffers -- the 512 x 512 phantom under all 12 solver / wavelet /
    transfer combinations at both noise levels (24 images, the default), or
    with --batch 12 at one noise level (1 % on even steps, 5 % on odd ones).
    The same images one at a time (deblur_solve) give the plain figures
    beside it."""
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
    x_true = I.phantom(M, 40, 20, SEED)
    bs = {nz: make_b(api, torch, M, x_true, psf, nz, 10_000 + SEED) for nz in NOISES}
    b_dev = {nz: torch.from_numpy(I.to_colmajor(b).ravel()).cuda() for nz, b in bs.items()}
    nb = args.batch
    xs = [torch.empty(M * M, dtype=torch.float64, device="cuda") for _ in range(nb)]

    def cases_of(s):
        """(noise, combination) of the images of step s: the 12 combinations at
        one noise level (1 % on even steps, 5 % on odd ones), or with
        --batch 24 all 24 cases of the workload."""
        noises = NOISES if args.batch == 24 else (NOISES[s % 2],)
        return [(nz, c) for nz in noises for c in COMBOS]

    def batch_dev(s):
        probs = [dict(b=b_dev[nz], psf=psf_dev, x=xs[j], m=M, psf_size=PSF_SIZE, solver=c[0], wavelet=c[1],
                      levels=LEVELS, transfer=c[2]) for j, (nz, c) in enumerate(cases_of(s))]
        return api.deblur_solve_batch_device(probs, precision="fp32", ctx=ctx, stream=stream.cuda_stream)

    for i in range(args.warmup):
        batch_dev(steps[i])
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times, par_in, seen = [], [], set()
    for i in range(args.warmup, total):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select exactly the timed steps
        res = batch_dev(steps[i])
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        for j, (nz, c) in enumerate(cases_of(steps[i])):
            name = case_name(c[0], c[1], c[2], nz)
            if name not in seen:                 # each case once, for the oracle comparison
                seen.add(name)
                par_in.append((name, xs[j].cpu().numpy(), res[j]["iters"], res[j]["mu"]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = ctx.stats()
    t_total_ms = max_over_ranks(sum(times), world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    images = nb * args.steps * world
    value = M * M * images / (t_total_ms / 1e3) / 1e6
    if args.only_timed:
        return {"metric": "deblurred Mpixel/s", "value": round(value, 4), "unit": "Mpixel/s",
                "ms_per_step": round(t_total_ms / args.steps, 3), "images_per_step": nb,
                "lsqr_ms_per_step": round(stats["lsqr_ms"] / args.steps, 2), "gpu_launches": int(stats["kernel_launches"])}, []
    parity = parity_summary(par_in, load_golden())

    # plain: the images of the first timed step, one deblur_solve each
    s0 = steps[args.warmup]
    plain_ms = 0.0
    for j, (nz, c) in enumerate(cases_of(s0)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.deblur_solve_device(b_dev[nz], psf_dev, M, PSF_SIZE, xs[j], c[0], c[1], LEVELS, c[2],
                                precision="fp32", ctx=ctx, stream=stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        plain_ms += e0.elapsed_time(e1)

    # e2e: the same batches through the host-buffer call (copies in and out
    # inside the timed region); --e2e-steps 0 skips it (profiling runs only)
    e2e_steps = args.steps if args.e2e_steps < 0 else min(args.steps, args.e2e_steps)
    e2e_ms = 0.0
    for i in range(e2e_steps):
        probs = [dict(b=bs[nz], psf=psf, solver=c[0], wavelet=c[1], levels=LEVELS, transfer=c[2])
                 for nz, c in cases_of(steps[args.warmup + i])]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.deblur_solve_batch(probs, precision="fp32", ctx=ctx, stream=stream.cuda_stream)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_value = M * M * nb * e2e_steps * world / (e2e_ms / 1e3) / 1e6 if e2e_steps else None

    peak, peak_kind = load_peaks()
    roofline = lsqr_roofline_all(stats, 4, 4, peak, peak_kind, t_total_ms, "m512",
                                 note=f"batched launches over the {nb} problems of a step, every level; the "
                                      f"vectors of {nb} m = 512 cycles (~{21 * nb} MB) exceed the 126 MB L2 "
                                      "only in part")
    line = {
        "metric": "deblurred Mpixel/s", "value": round(value, 4), "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_total_ms / args.steps, 3),
        "images_per_step": nb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic phantoms (inputs module), b = A x_true by the library's blur + seeded noise, "
                "rounded to float32",
        "config": workload_desc(args.batch),
        "images_per_s": round(images / (t_total_ms / 1e3), 4),
        "plain": {"images_per_s": round(nb / (plain_ms / 1e3), 4),
                  "mpixel_per_s": round(M * M * nb / (plain_ms / 1e3) / 1e6, 4),
                  "ms_per_image": round(plain_ms / nb, 1), "call": "deblur_solve, one image at a time"},
        "e2e": None if e2e_value is None else
               {"value": round(e2e_value, 4), "unit": "Mpixel/s", "steps": e2e_steps,
                "h2d_bytes_per_step": nb * (M * M * 8 + PSF_SIZE * PSF_SIZE * 8),
                "d2h_bytes_per_step": nb * (M * M * 8 + LEVELS * 16)},
        "gpu_launches": int(stats["kernel_launches"]),
        "roofline": roofline,
        "oracle_parity": parity,
        "clocks": clk,
        "counts": {"lsqr_launches": int(stats["lsqr_launches"]), "gcv_calls": int(stats["gcv_calls"]),
                   "outer_iterations": int(stats["outer_iterations"])},
        "step_split": {"lsqr_ms_per_step": round(stats["lsqr_ms"] / args.steps, 2),
                       "gcv_ms_per_step": round(stats.get("gcv_ms", 0.0) / args.steps, 2),
                       "note": "GCV time is host wall time summed over the worker threads"},
    }
    if world == 1 and args.large_steps > 0:
        line["large"] = run_large(api, torch, ctx, args.large_steps, flush, peak, peak_kind)
    if world == 1 and args.forms:
        line["serving"] = run_serving_m512(api, ctx, bs, psf)
    return line, [n for n, _, _, _ in par_in]


def lsqr_roofline_all(stats, elem, x_elem, peak, peak_kind, t_total_ms, key, note):
    """achieved = algorithmic bytes of every k_lsqr launch of the timed
    region / their CUDA-event time (event pair around each launch on the
    solve's stream)."""
    bytes_alg = (stats["lsqr_pixel_iters_irls"] * lsqr_bytes_per_pixel_iter(elem, x_elem, True)
                 + stats["lsqr_pixel_iters_other"] * lsqr_bytes_per_pixel_iter(elem, x_elem, False))
    launches = max(1, stats["lsqr_launches"])
    ms = stats["lsqr_ms"]
    achieved = (bytes_alg / launches) / ((ms / launches) / 1e3) / 1e9 if ms > 0 else 0.0
    traffic, scope = lsqr_traffic(key, (stats["lsqr_pixel_iters_irls"] + stats["lsqr_pixel_iters_other"]) / launches)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_scope": scope,
            "algorithmic_bytes_per_launch": round(bytes_alg / launches),
            "kernel": "k_lsqr (persistent cooperative LSQR), every launch of the timed region",
            "launches": int(stats["lsqr_launches"]), "peak_kind": peak_kind,
            "lsqr_share_of_step": round(ms / t_total_ms, 4) if t_total_ms else None, "note": note}


def run_serving_m512(api, ctx, bs, psf):
    """Poisson arrivals of the 24 cases (12 combinations x 2 noise levels, each
    twice) at 80 % of the server's saturated rate, measured first with every
    request queued at once; p50 / p99 latency from submit to completion."""
    reqs = [(bs[nz], c) for nz in NOISES for c in COMBOS]
    srv = api.Server(max_resident=len(reqs), max_m=M, ctx=api.Context(0))
    t0 = time.perf_counter()
    tks = [srv.submit(b, psf, c[0], c[1], LEVELS, c[2]) for b, c in reqs]
    lat_all = [srv.poll(tk)[1] for tk in tks]
    t_sat = time.perf_counter() - t0
    srv.close()
    sat = len(reqs) / t_sat
    rng = np.random.default_rng(2026)
    order = [i % len(reqs) for i in range(2 * len(reqs))]
    gaps = rng.exponential(1.0 / (0.8 * sat), size=len(order))
    srv = api.Server(max_resident=len(reqs), max_m=M, ctx=api.Context(0))
    t0 = time.perf_counter()
    tks, t_next = [], 0.0
    for k, i in enumerate(order):
        t_next += gaps[k]
        while time.perf_counter() - t0 < t_next:
            time.sleep(0.0005)
        b, c = reqs[i]
        tks.append(srv.submit(b, psf, c[0], c[1], LEVELS, c[2]))
    lat = [srv.poll(tk)[1] for tk in tks]
    t_p = time.perf_counter() - t0
    srv.close()
    return {"saturated_images_per_s": round(sat, 4), "requests": len(reqs),
            "all_queued_p50_ms": round(float(np.percentile(lat_all, 50)), 1),
            "poisson": {"rate_per_s": round(0.8 * sat, 3), "requests": len(order),
                        "images_per_s": round(len(order) / t_p, 4),
                        "p50_ms": round(float(np.percentile(lat, 50)), 1),
                        "p99_ms": round(float(np.percentile(lat, 99)), 1)}}


def lsqr_roofline(stats, elem, x_elem, peak, peak_kind, t_total_ms, key, note):
    """achieved = algorithmic bytes of the finest-level k_lsqr launches /
    their CUDA-event time (the library records an event pair around every
    LSQR launch on the solve's stream when profiling is on)."""
    bytes_alg = (stats["lsqr_fine_pixel_iters_irls"] * lsqr_bytes_per_pixel_iter(elem, x_elem, True)
                 + stats["lsqr_fine_pixel_iters_other"] * lsqr_bytes_per_pixel_iter(elem, x_elem, False))
    launches = max(1, stats["lsqr_fine_launches"])
    ms = stats["lsqr_fine_ms"]
    achieved = (bytes_alg / launches) / ((ms / launches) / 1e3) / 1e9 if ms > 0 else 0.0
    traffic, scope = lsqr_traffic(key, (stats["lsqr_fine_pixel_iters_irls"] + stats["lsqr_fine_pixel_iters_other"])
                                  / launches)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_scope": scope,
            "algorithmic_bytes_per_launch": round(bytes_alg / launches),
            "kernel": "k_lsqr (persistent cooperative LSQR), finest-level launches",
            "launches": int(stats["lsqr_fine_launches"]), "peak_kind": peak_kind,
            "lsqr_share_of_step": round(stats["lsqr_ms"] / t_total_ms, 4) if t_total_ms else None,
            "note": note}


def run_large(api, torch, ctx, nsteps, flush, peak, peak_kind):
    """A few timed solves of the large-image workload: m = 2048, Gaussian
    sigma = 6 on 31 x 31 or the 21-pixel motion blur at 30 degrees, 1 %
    noise, BF16 storage, 5-level Db4 cycles; with the finest-level k_lsqr
    roofline."""
    from paper_2608_17123_b300 import inputs as I
    m = LARGE_M
    R = int(round(40 * math.sqrt(m / 512)))
    x_true = I.phantom(m, R, R // 2, SEED)
    psfs = {"gauss31": I.gaussian_psf(6.0, 31), "motion21": I.motion_psf(21.0, 30.0, 21)}
    bdev, pdev = {}, {}
    for name, p in psfs.items():
        b = make_b(api, torch, m, x_true, p, 0.01, 10_000 + SEED)
        bdev[name] = torch.from_numpy(I.to_colmajor(b).ravel()).cuda()
        pdev[name] = torch.from_numpy(I.to_colmajor(p).ravel()).cuda()
    xd = torch.empty(m * m, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def solve(k):
        pname, solver, transfer = LARGE_CASES[k % len(LARGE_CASES)]
        return api.deblur_solve_device(bdev[pname], pdev[pname], m, psfs[pname].shape[0], xd, solver, "db4", 5,
                                       transfer, precision="bf16", ctx=ctx, stream=stream.cuda_stream)

    solve(0)                                   # warm-up (first launches of the size class)
    torch.cuda.synchronize()
    ctx.reset_stats()
    times, rres, cases = [], [], []
    for k in range(nsteps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = solve(k)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        x = I.from_colmajor(xd.cpu().numpy(), m)
        rres.append(float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true)))
        cases.append({"case": "-".join(LARGE_CASES[k % len(LARGE_CASES)]), "ms": round(times[-1], 1),
                      "iters": r["iters"], "rre_vs_phantom": round(rres[-1], 4)})
    stats = ctx.stats()
    t = sum(times)
    return {"workload": f"m{m}_db4_5level_bf16", "m": m, "steps": nsteps, "ms_per_step": round(t / nsteps, 1),
            "value": round(m * m * nsteps / (t / 1e3) / 1e6, 4), "unit": "Mpixel/s",
            "precision": "bf16 storage (image, planes, Krylov vectors), fp32 iterate and LSQR correction",
            "cases": cases,
            "roofline": lsqr_roofline(stats, 2, 4, peak, peak_kind, t, "large",
                                      note="BF16 LSQR vectors of a 2048 x 2048 level: ~80-90 MB, near the "
                                           "L2 size"),
            "step_split": {"lsqr_ms_per_step": round(stats["lsqr_ms"] / nsteps, 1),
                           "gcv_ms_per_step": round(stats.get("gcv_ms", 0.0) / nsteps, 1)}}


# ------------------------------------------------------------------ oracle sample
def gcv_calls(solver, level, outer):
    """GCV estimates a level makes under the schedule of Sec. 3 (3-level
    cycles): IRLS re-estimates at every outer iteration, except on the fine
    level, where it estimates at k = 0 and k = 3; MM and SB at k = 0, 1, 2."""
    if solver == "irls":
        if level == 0 and LEVELS >= 3:
            return 1 + (1 if outer > 3 else 0)
        return outer
    return min(3, outer)


def sample_unit_costs(levels_to_time, lsqr_iters=(8, 16, 32)):
    """Seconds per LSQR iteration and per GCV call of the FP64 oracle on the
    m = 512 workload's own level problems (Db4 hierarchy, 1 % noise): LSQR on
    the MM form (shift from the Tikhonov-free start), GCV as IRLS calls it
    (the weighted pair with the weights of the level's restricted data, the
    k = 40, 80, 160 doubling)."""
    from oracle import operators as O
    from oracle import solvers as S
    from paper_2608_17123_b300 import inputs as I
    g = I.gaussian_factor(SIGMA, PSF_SIZE)
    A = O.KronOp.from_factors(M, g, g)
    x_true = I.phantom(M, 40, 20, SEED)
    b = I.add_noise(A.apply(x_true), I.noise_direction(M, 10_000 + SEED), 0.01)
    As, bs = [A], [b]
    for _ in range(LEVELS - 1):
        As.append(As[-1].coarsen("db4"))
        bs.append(O.restrict(bs[-1], "db4"))
    t_lsqr, t_gcv = {}, {}
    for lvl in range(LEVELS):
        mm = As[lvl].m
        z = (np.zeros((mm - 1, mm)), np.zeros((mm, mm - 1)))
        sub = S.Subproblem(As[lvl], bs[lvl], c=z)
        its = lsqr_iters[lvl]
        t = time.perf_counter()
        _, k = sub.solve(1e-3, np.zeros((mm, mm)), S.opts_with(lsqr_maxit=its, lsqr_atol=0, lsqr_btol=0))
        t_lsqr[lvl] = (time.perf_counter() - t) / max(k, 1)
        if lvl in levels_to_time:
            w = S.irls_weights(*O.L_apply(bs[lvl] / (2.0 ** lvl)), 0.03)
            t = time.perf_counter()
            S.Subproblem(As[lvl], bs[lvl], weights=w).gcv(S.opts_with())
            t_gcv[lvl] = time.perf_counter() - t
    return t_lsqr, t_gcv


def _unit_costs_worker(q, levels_to_time):
    q.put(sample_unit_costs(levels_to_time))


def unit_costs_with_threads(threads, levels_to_time):
    """sample_unit_costs in a fresh process whose BLAS uses `threads`
    threads (the variables must be set before numpy loads)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = str(threads)
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_unit_costs_worker, args=(q, tuple(levels_to_time)))
        p.start()
        res = q.get()
        p.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res


def model_solve_seconds(t_lsqr, t_gcv, golden, names):
    """Oracle seconds per solve of the given cases: the oracle's own recorded
    work counts (outer iterations and LSQR iterations per level, from its
    stored runs of these cases) times the measured unit costs."""
    tot = 0.0
    for nm in names:
        c = golden["cases"][nm]
        for l in range(LEVELS):
            tot += c["inner"][l] * t_lsqr[l] + gcv_calls(c["solver"], l, c["iters"][l]) * t_gcv[l]
    return tot / len(names)


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(names):
    """The cpu_baseline of our line: the oracle's unit costs on this host
    (1 BLAS thread and all cores), scaled to Mpixel/s with the oracle's
    recorded work counts of the timed steps' cases."""
    golden = load_golden()
    if golden is None:
        return None
    names = [n for n in names if n in golden["cases"]]
    out = {}
    t0 = time.perf_counter()
    for threads in (1, os.cpu_count() or 1):
        tl, tg = unit_costs_with_threads(threads, (0, 1, 2))
        sec = model_solve_seconds(tl, tg, golden, names)
        out[threads] = (M * M / sec / 1e6, sec, tl, tg)
    elapsed = time.perf_counter() - t0
    nc = os.cpu_count() or 1
    v_all, sec_all, tl, tg = out[nc]
    v1, sec1, _, _ = out[1]
    wall = [golden["cases"][n].get("oracle_wall_s_one_thread") for n in names]
    return {"value": v_all, "unit": "Mpixel/s", "cores": nc, "kind": "oracle",
            "cpu": cpu_model(),
            "one_thread": {"value": v1, "seconds_per_solve": round(sec1, 1)},
            "seconds_per_solve": round(sec_all, 1),
            "sample": (f"FP64 oracle on this host: seconds per LSQR iteration on the 512/256/128 levels "
                       f"({tl[0]*1e3:.1f}/{tl[1]*1e3:.1f}/{tl[2]*1e3:.1f} ms with {nc} BLAS threads) and per "
                       f"IRLS-type GCV call ({tg[0]:.2f}/{tg[1]:.2f}/{tg[2]:.2f} s), times the oracle's own "
                       f"recorded counts (outer and LSQR iterations per level) of the {len(names)} timed cases; "
                       f"{elapsed:.0f} s of CPU work"),
            "full_solve_reference_s": {"note": "complete single-thread oracle solves of the same cases, timed when "
                                               "the stored results were written (another host)",
                                       "median": float(np.median([w for w in wall if w])) if any(wall) else None}}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: step s times LSQR iterations on the
    three level problems and one GCV call on level s mod 3 (the last step
    also on any level no earlier step reached; a bounded sample of the
    workload's solves); the Mpixel/s value scales the measured unit costs by
    the oracle's recorded counts of the workload's cases."""
    if rank != 0:
        return None
    golden = load_golden()
    if golden is None:
        return {"impl": "reference", "unavailable": "stored oracle counts (tests/golden/m512_oracle) missing"}
    names = [case_name(c[0], c[1], c[2], nz) for nz in NOISES for c in COMBOS]
    names = [n for n in names if n in golden["cases"]]
    for s in range(args.warmup):
        sample_unit_costs((s % LEVELS,), lsqr_iters=(2, 4, 8))
    tl_acc = {l: [] for l in range(LEVELS)}
    tg_acc = {l: [] for l in range(LEVELS)}
    t_steps = []
    for s in range(args.steps):
        # the level of this step; the last step also takes every level no
        # earlier step reached (runs of fewer than LEVELS steps)
        lv = [s % LEVELS]
        if s == args.steps - 1:
            lv += [l for l in range(LEVELS) if not tg_acc[l] and l not in lv]
        t0 = time.perf_counter()
        tl, tg = sample_unit_costs(tuple(lv))
        t_steps.append(time.perf_counter() - t0)
        for l in range(LEVELS):
            tl_acc[l].append(tl[l])
        for l, v in tg.items():
            tg_acc[l].append(v)
    tl = {l: statistics.median(v) for l, v in tl_acc.items()}
    tg = {l: statistics.median(v) if v else float("nan") for l, v in tg_acc.items()}
    sec = model_solve_seconds(tl, tg, golden, names)
    value = M * M / sec / 1e6
    nc = os.cpu_count() or 1
    cb = {"value": value, "unit": "Mpixel/s", "cores": nc, "kind": "oracle", "cpu": cpu_model(),
          "sample": (f"{args.steps} steps, each: LSQR iterations on the 512/256/128 level problems and one GCV "
                     f"call on one level (the level cycles with the step); unit costs (medians) "
                     f"{tl[0]*1e3:.1f}/{tl[1]*1e3:.1f}/{tl[2]*1e3:.1f} ms per LSQR iteration, "
                     f"{tg[0]:.2f}/{tg[1]:.2f}/{tg[2]:.2f} s per GCV call, scaled by the oracle's recorded counts "
                     f"of the cases -> {sec:.0f} s per solve"),
          "seconds_per_solve": round(sec, 1)}
    ms_step = 1e3 * statistics.mean(t_steps)
    return {"metric": "deblurred Mpixel/s", "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(args.batch), "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ batched / served workloads
def uneven_requests(count, sizes, seed, noise_range=(0.01, 0.01)):
    """`count` requests of uneven size: m uniform over `sizes`, Gaussian PSF
    sigma ~ U[1.5, 6] on S = min(31, 2 ceil(3 sigma) + 1), noise level
    uniform over noise_range, solver / wavelet / transfer each uniform,
    3-level cycles (up to log2(m) - 6 levels for m < 512), phantoms with
    40 sqrt(m / 512) rectangles and half as many disks. Returns a list of
    dicts (b without noise rounding: the FP32 path rounds on the device)."""
    from paper_2608_17123_b300 import inputs as I
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(count):
        m = int(rng.choice(sizes))
        sigma = float(rng.uniform(1.5, 6.0))
        S_ = min(31, 2 * int(math.ceil(3 * sigma)) + 1)
        solver = ("irls", "mm", "sb")[int(rng.integers(3))]
        wavelet = ("haar", "db4")[int(rng.integers(2))]
        transfer = ("X", "D")[int(rng.integers(2))]
        noise = float(rng.uniform(*noise_range))
        R = max(4, int(round(40 * math.sqrt(m / 512))))
        reqs.append(dict(m=m, sigma=sigma, S=S_, solver=solver, wavelet=wavelet, transfer=transfer,
                         noise=noise, levels=3, seed=1000 + k, nr=R, nd=R // 2))
    return reqs


def materialise(api, torch, reqs):
    from paper_2608_17123_b300 import inputs as I
    out = []
    for r in reqs:
        psf = I.gaussian_psf(r["sigma"], r["S"])
        x_true = I.phantom(r["m"], r["nr"], r["nd"], r["seed"])
        b = make_b(api, torch, r["m"], x_true, psf, r["noise"], 30_000 + r["seed"])
        out.append(dict(b=b, psf=psf, solver=r["solver"], wavelet=r["wavelet"], levels=r["levels"],
                        transfer=r["transfer"], x_true=x_true))
    return out


def run_batch_workload(args):
    """64 images of uneven size (m in {128, 256, 512, 1024, 2048}, seed 7),
    mixed PSFs, solvers, wavelets and transfers, FP32: one deblur_solve_batch
    call against the same 64 solves one at a time (deblur_solve), images/s
    of each and the largest difference between the two reconstructions."""
    import torch
    from paper_2608_17123_b300 import api
    reqs = materialise(api, torch, uneven_requests(args.batch_images, (128, 256, 512, 1024, 2048), 7))
    ctx = api.Context(0)
    api.deblur_solve(reqs[0]["b"], reqs[0]["psf"], reqs[0]["solver"], reqs[0]["wavelet"], 3, reqs[0]["transfer"],
                     precision="fp32", ctx=ctx)   # warm-up (module load, first launches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [api.deblur_solve(r["b"], r["psf"], r["solver"], r["wavelet"], 3, r["transfer"], precision="fp32",
                              ctx=ctx) for r in reqs]
    t_plain = time.perf_counter() - t0
    probs = [{k: r[k] for k in ("b", "psf", "solver", "wavelet", "levels", "transfer")} for r in reqs]
    t0 = time.perf_counter()
    batched = api.deblur_solve_batch(probs, precision="fp32", ctx=ctx)
    t_batch = time.perf_counter() - t0
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    pix = sum(r["b"].size for r in reqs)
    n = len(reqs)
    return {"workload": "batch64_uneven_m128-2048_mixed", "images": n, "megapixels": round(pix / 1e6, 3),
            "sizes": sorted(set(r["b"].shape[0] for r in reqs)),
            "plain": {"images_per_s": round(n / t_plain, 4), "mpixel_per_s": round(pix / t_plain / 1e6, 4),
                      "s": round(t_plain, 2)},
            "batched": {"images_per_s": round(n / t_batch, 4), "mpixel_per_s": round(pix / t_batch / 1e6, 4),
                        "s": round(t_batch, 2)},
            "speedup": round(t_plain / t_batch, 3),
            "max_rel_diff_batched_vs_plain": max(rel(b["x"], p["x"]) for b, p in zip(batched, plain)),
            "io": "host buffers (each call copies its inputs in and its result out)", "precision": "fp32"}


def run_serve_workload(args):
    """Continuous-batching server under a Poisson request stream: requests of
    m in {256, 512, 1024} (mixed PSFs, solvers, wavelets, transfers, noise
    1-5 %), the rate swept over fractions of the plain one-at-a-time
    throughput of the same requests; images/s delivered and p50/p99 latency
    (arrival to completion) at each rate, and the largest difference of a
    served result from its one-at-a-time solve."""
    import torch
    from paper_2608_17123_b300 import api
    reqs = materialise(api, torch, uneven_requests(args.serve_requests, (256, 512, 1024), 11, (0.01, 0.05)))
    ctx = api.Context(0)
    api.deblur_solve(reqs[0]["b"], reqs[0]["psf"], reqs[0]["solver"], reqs[0]["wavelet"], 3, reqs[0]["transfer"],
                     precision="fp32", ctx=ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [api.deblur_solve(r["b"], r["psf"], r["solver"], r["wavelet"], 3, r["transfer"], precision="fp32",
                              ctx=ctx) for r in reqs]
    t_plain = time.perf_counter() - t0
    plain_rate = len(reqs) / t_plain
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    points = []
    worst = 0.0
    for frac in args.serve_rates:
        rate = frac * plain_rate
        rng = np.random.default_rng(int(1000 * frac))
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        srv = api.Server(max_resident=args.serve_slots, max_m=1024, ctx=ctx)
        t0 = time.perf_counter()
        tks, t_next = [], 0.0
        for k, r in enumerate(reqs):
            t_next += gaps[k]
            while time.perf_counter() - t0 < t_next:
                time.sleep(0.0005)
            tks.append(srv.submit(r["b"], r["psf"], r["solver"], r["wavelet"], 3, r["transfer"]))
        res = [srv.poll(t) for t in tks]
        t_all = time.perf_counter() - t0
        srv.close()
        lat = [l for _, l in res]
        worst = max(worst, max(rel(q["x"], p["x"]) for (q, _), p in zip(res, plain)))
        points.append({"offered_fraction_of_plain": frac, "offered_per_s": round(rate, 3),
                       "delivered_images_per_s": round(len(reqs) / t_all, 4),
                       "p50_ms": round(float(np.percentile(lat, 50)), 1),
                       "p99_ms": round(float(np.percentile(lat, 99)), 1)})
    return {"workload": "serve_poisson_m256-1024_mixed", "requests_per_point": len(reqs),
            "slots": args.serve_slots, "plain_images_per_s": round(plain_rate, 4),
            "plain_p50_ms": round(1e3 * t_plain / len(reqs), 1), "points": points,
            "max_rel_diff_served_vs_plain": worst, "precision": "fp32"}


# ------------------------------------------------------------------ single LSQR launches
def run_lsqr_probe(args):
    """Four LSQR solves of one level-0 MM subproblem (gamma = 1e-3, 100
    iterations, stopping tolerances off) on an m x m phantom with the given
    PSF, FP32, autotuning off: one k_lsqr launch each. The profiler
    recipes of profiles/ capture the fourth launch (-k regex:k_lsqr -s 3 -c 1)."""
    import torch
    from paper_2608_17123_b300 import api
    from paper_2608_17123_b300 import inputs as I
    m = args.lsqr_m
    psf = I.gaussian_psf(*{"gauss31": (6.0, 31), "gauss15": (3.0, 15)}[args.lsqr_psf])
    ctx = api.Context(0)
    ctx.set_autotune(False)
    if args.lsqr_prec == "bf16":
        # BF16 storage is reachable through the solve only: a single-level MM
        # cycle of three outer iterations, one k_lsqr launch each
        x_true = I.phantom(m, 40, 20, 6)
        b = make_b(api, torch, m, x_true, psf, 0.01, 777)
        bd = torch.from_numpy(I.to_colmajor(b).ravel()).cuda()
        pd = torch.from_numpy(I.to_colmajor(psf).ravel()).cuda()
        xd = torch.empty(m * m, dtype=torch.float64, device="cuda")
        ctx.set_profiling(True)
        r = api.deblur_solve_device(bd, pd, m, psf.shape[0], xd, "mm", "haar", 1, "I", precision="bf16", ctx=ctx,
                                    kmax=3, gamma_fixed=1e-3, fine_direct=args.lsqr_direct)
        st = ctx.stats()
        ctx.close()
        alg = (st["lsqr_pixel_iters_other"]) * lsqr_bytes_per_pixel_iter(2, 4, False)
        return {"probe": "lsqr", "m": m, "psf": args.lsqr_psf, "precision": "bf16", "direct": args.lsqr_direct,
                "launches": st["lsqr_launches"],
                "pixel_iterations": st["lsqr_pixel_iters_other"], "ms": round(st["lsqr_ms"], 3),
                "algorithmic_gb_s": round(alg / st["lsqr_ms"] / 1e6, 1)}
    xt = torch.from_numpy(I.to_colmajor(I.phantom(m, 40, 20, 6)).ravel()).to("cuda", torch.float32)
    b = torch.empty_like(xt)
    api.apply_blur(psf, m, xt, b, ctx=ctx)
    x0 = 0.9 * xt
    c = torch.zeros(2 * m * m, device="cuda", dtype=torch.float32)
    xo = torch.empty_like(xt)
    for _ in range(3):
        api.lsqr_solve(psf, m, "mm", 1e-3, b, x0, c, None, xo, ctx=ctx, lsqr_maxit=100, lsqr_atol=0.0, lsqr_btol=0.0,
                       fine_direct=args.lsqr_direct)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    its = api.lsqr_solve(psf, m, "mm", 1e-3, b, x0, c, None, xo, ctx=ctx, lsqr_maxit=100, lsqr_atol=0.0,
                         lsqr_btol=0.0, fine_direct=args.lsqr_direct)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    alg = (its + 1) * m * m * lsqr_bytes_per_pixel_iter(4, 4, False)
    return {"probe": "lsqr", "m": m, "psf": args.lsqr_psf, "direct": args.lsqr_direct, "iterations": its,
            "ms": round(ms, 3),
            "us_per_iteration": round(1e3 * ms / its, 2), "algorithmic_gb_s": round(alg / ms / 1e6, 1)}


def run_one_solve(args):
    """One m = 512 image of the benchmark workload (one solver / wavelet /
    transfer combination at one noise level) by the plain call, after one
    untimed solve of the same image: the command the per-kernel launch lists
    of profiles/ are taken on (about 5-9 K launches)."""
    import torch
    from paper_2608_17123_b300 import api
    from paper_2608_17123_b300 import inputs as I
    solver, wavelet, transfer = args.combo.split("-")
    ctx = api.Context(0)
    ctx.set_profiling(True)
    psf = I.gaussian_psf(SIGMA, PSF_SIZE)
    psf_dev = torch.from_numpy(I.to_colmajor(psf).ravel()).cuda()
    x_true = I.phantom(M, 40, 20, SEED)
    b = make_b(api, torch, M, x_true, psf, args.noise, 10_000 + SEED)
    b_dev = torch.from_numpy(I.to_colmajor(b).ravel()).cuda()
    xd = torch.empty(M * M, dtype=torch.float64, device="cuda")
    run = lambda: api.deblur_solve_device(b_dev, psf_dev, M, PSF_SIZE, xd, solver, wavelet, LEVELS, transfer,
                                          precision="fp32", ctx=ctx)
    run()
    torch.cuda.synchronize()
    ctx.reset_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = run()
    e1.record()
    e1.synchronize()
    st = ctx.stats()
    ctx.close()
    return {"probe": "solve", "m": M, "combo": args.combo, "noise": args.noise, "ms": round(e0.elapsed_time(e1), 2),
            "iters": r["iters"], "launches": st["kernel_launches"], "lsqr_ms": round(st["lsqr_ms"], 2)}


# ------------------------------------------------------------------ phantom study
def ssim(x, y, L=None, win=11, sigma=1.5):
    """Structural similarity index (Wang, Bovik, Sheikh, Simoncelli 2004):
    local means, variances and covariance over Gaussian-weighted win x win
    windows (standard deviation sigma, weights summing to 1), the index
    ((2 mu_x mu_y + c1)(2 s_xy + c2)) / ((mu_x^2 + mu_y^2 + c1)(s_x^2 + s_y^2 + c2))
    with c1 = (0.01 L)^2, c2 = (0.03 L)^2, averaged over every window that
    lies inside the image. L: dynamic range (default: that of x)."""
    from scipy.signal import convolve2d
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if L is None:
        L = float(x.max() - x.min()) or 1.0
    r = win // 2
    g = np.exp(-(np.arange(-r, r + 1) ** 2) / (2.0 * sigma * sigma))
    w = np.outer(g, g)
    w /= w.sum()
    f = lambda a: convolve2d(a, w, mode="valid")
    mx, my = f(x), f(y)
    sxx = f(x * x) - mx * mx
    syy = f(y * y) - my * my
    sxy = f(x * y) - mx * my
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    smap = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(smap.mean())


def run_phantom_study(args):
    """The paper's experiments (Sec. 5) on synthetic phantoms: 64 x 64
    two-level and 128 x 128 three-level V-cycles, Gaussian blur sigma = 3.5
    and 4.5, 1 % noise; IRLS, MM and SB, each single-level (Approach I, at
    64 x 64) and with HWT-D, HWT-X, DWT-D, DWT-X. Reports RRE, SSIM, device
    time and outer iterations per level for every run."""
    import torch
    from paper_2608_17123_b300 import api
    from paper_2608_17123_b300 import inputs as I
    ctx = api.Context(0)
    rows = []
    for m, levels, nr, nd in ((64, 2, 12, 6), (128, 3, 24, 12)):
        x_true = I.phantom(m, nr, nd, SEED)
        for sigma in (3.5, 4.5):
            S_ = 2 * int(math.ceil(3 * sigma)) + 1
            psf = I.gaussian_psf(sigma, S_)
            b = make_b(api, torch, m, x_true, psf, 0.01, 20_000 + m)
            runs = [("I", "haar", 1)] if levels == 2 else []
            runs += [(t, w, levels) for w in ("haar", "db4") for t in ("D", "X")]
            for solver in ("irls", "mm", "sb"):
                for transfer, wavelet, lv in runs:
                    api.deblur_solve(b, psf, solver, wavelet, lv, transfer, precision="fp64", ctx=ctx)  # warm
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    r = api.deblur_solve(b, psf, solver, wavelet, lv, transfer, precision="fp64", ctx=ctx)
                    dt = time.perf_counter() - t0
                    name = "I" if lv == 1 else ("HWT" if wavelet == "haar" else "DWT") + "-" + transfer
                    rows.append({"m": m, "sigma": sigma, "solver": solver, "method": name,
                                 "rre": round(float(np.linalg.norm(r["x"] - x_true) / np.linalg.norm(x_true)), 4),
                                 "ssim": round(ssim(x_true, r["x"]), 4), "ms": round(dt * 1e3, 1),
                                 "iters": r["iters"]})
    ctx.close()
    return {"study": "phantom_multilevel", "precision": "fp64", "psf": "gaussian, S = 2 ceil(3 sigma) + 1",
            "noise": "1%", "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=-1, help="-1: every timed step")
    ap.add_argument("--large-steps", type=int, default=3)
    ap.add_argument("--batch", type=int, default=24, choices=[12, 24],
                    help="images per step: the 12 combinations at one noise level, or all 24 cases")
    ap.add_argument("--only-timed", action="store_true",
                    help="stop after the timed steps (profiling runs: no plain, e2e, parity, large, serving "
                         "or CPU measurement)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the serving measurement")
    ap.add_argument("--lsqr-m", type=int, default=2048)
    ap.add_argument("--lsqr-psf", default="gauss31", choices=["gauss31", "gauss15"])
    ap.add_argument("--lsqr-prec", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--lsqr-direct", type=int, default=1, choices=[0, 1],
                    help="level-0 blur of the probe: 1 direct (TMA windows), 0 band form")
    ap.add_argument("--combo", default="irls-haar-X", help="solve probe: solver-wavelet-transfer")
    ap.add_argument("--noise", type=float, default=0.01, help="solve probe: noise level")
    ap.add_argument("--workload", default="m512", choices=["m512", "batch", "serve", "study", "lsqr", "solve"],
                    help="m512: the benchmark line; batch: 64 uneven images batched vs one at a time; "
                         "serve: Poisson request stream against the server; study: the phantom study of "
                         "the paper's experiments; lsqr: four single-level LSQR launches (profiling); solve: "
                         "one plain solve of one m = 512 case (profiling)")
    ap.add_argument("--batch-images", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 1.0, 2.0, 4.0])
    args = ap.parse_args()
    if args.workload != "m512":
        fn = {"batch": run_batch_workload, "serve": run_serve_workload, "study": run_phantom_study,
              "lsqr": run_lsqr_probe, "solve": run_one_solve}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return
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
    line, names = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and not args.only_timed:
            line["cpu_baseline"] = oracle_sample(names)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
