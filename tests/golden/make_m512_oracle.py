#!/usr/bin/env python
"""Writes the FP64 oracle's results for the m = 512 workload into
tests/golden/m512_oracle/ (one .npz per case plus index.json).

Workload: a 512 x 512 piecewise-constant phantom (40 rectangles, 20 disks,
seed 0), Gaussian PSF sigma = 3 on 15 x 15 (sum 1), b = A x_true + e with e
at 1 % and 5 % of ||A x_true|| (Sec. 5 defines the noise relative to the
blurred image), rounded to float32 (the storage precision of the GPU path,
which then sees exactly the same input); 3-level V-cycles (Alg. 4) of IRLS,
MM and SB (Alg. 1-3) with the Haar and Daubechies-4 wavelets under both
transfer strategies (Approach X: the solution; Approach D: the solver's
auxiliary iterates), gamma by GCV on every level (Sec. 3).

Each case stores: gamma (mu or lambda) per level, outer and LSQR iteration
counts per level, ||x||, x at 16384 fixed pixels (sampled once, seed 512),
the wall time of the plain oracle solve (one BLAS thread; several cases run
at once, one per core),
and the oracle's own sensitivity to rounding ("spread"): the largest change
of x, gamma and the outer counts over two reruns with float32 unit-roundoff
noise injected into every operator output (the model of FP32 storage that
tests/perturb.py implements).

This script calls only oracle/ and the input generator. It takes about an
hour of CPU on 8 cores (every case runs three full solves); cases already
written are skipped, so it can be resumed.

    python tests/golden/make_m512_oracle.py [--jobs 8] [--cases irls-haar-X-0.01,...]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "m512_oracle")

M, SIGMA, PSF_SIZE, LEVELS, SEED = 512, 3.0, 15, 3, 0
N_RECT, N_DISK = 40, 20
NOISES = (0.01, 0.05)
COMBOS = [(s, w, t) for s in ("irls", "mm", "sb") for w in ("haar", "db4") for t in ("X", "D")]
N_SAMPLES, SAMPLE_SEED = 16384, 512
PERTURB_SEEDS = (12345, 777)


def case_name(solver, wavelet, transfer, noise):
    return f"{solver}-{wavelet}-{transfer}-{noise:g}"


def all_cases():
    return [(s, w, t, nz) for nz in NOISES for (s, w, t) in COMBOS]


def problem(noise):
    """(A, b rounded to float32, x_true) of the workload at one noise level."""
    import numpy as np
    from oracle import operators as O
    from paper_2608_17123_b300 import inputs as I
    g = I.gaussian_factor(SIGMA, PSF_SIZE)
    A = O.KronOp.from_factors(M, g, g)
    x_true = I.phantom(M, N_RECT, N_DISK, SEED)
    b = I.add_noise(A.apply(x_true), I.noise_direction(M, 10_000 + SEED), noise)
    return A, b.astype(np.float32).astype(np.float64), x_true


def run_case(spec):
    solver, wavelet, transfer, noise = spec
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    from oracle import solvers as S
    from perturb import noisy
    name = case_name(*spec)
    path = os.path.join(OUT, name + ".npz")
    if os.path.exists(path):
        return name, 0.0
    t0 = time.time()
    A, b, x_true = problem(noise)
    t1 = time.time()
    r0 = S.mgm(b, A, solver, wavelet, LEVELS, transfer)
    wall = time.time() - t1
    reruns = [noisy(lambda: S.mgm(b, A, solver, wavelet, LEVELS, transfer), "fp32", s) for s in PERTURB_SEEDS]
    x0 = r0["x"]
    idx = np.load(os.path.join(OUT, "sample_index.npy"))
    xs = x0.T.reshape(-1)[idx]          # column-major vec(X), element (r, c) at r + c*m
    nx = float(np.linalg.norm(x0))
    spread_x = max(float(np.linalg.norm(q["x"] - x0) / nx) for q in reruns)
    spread_mu = [max(abs(q["mu"][i] - r0["mu"][i]) / r0["mu"][i] for q in reruns) for i in range(LEVELS)]
    spread_it = [max(abs(q["iters"][i] - r0["iters"][i]) for q in reruns) for i in range(LEVELS)]
    rre = float(np.linalg.norm(x0 - x_true) / np.linalg.norm(x_true))
    tmp = path + ".tmp.npz"
    np.savez(tmp, x_samples=xs.astype(np.float32), mu=np.array(r0["mu"], dtype=np.float64),
             iters=np.array(r0["iters"], dtype=np.int32), inner=np.array(r0["inner"], dtype=np.int32),
             xnorm=np.float64(nx), rre=np.float64(rre), spread_x=np.float64(spread_x),
             spread_mu=np.array(spread_mu), spread_it=np.array(spread_it, dtype=np.int32),
             rerun_mu=np.array([q["mu"] for q in reruns]), rerun_iters=np.array([q["iters"] for q in reruns]),
             oracle_wall_s=np.float64(wall))
    os.replace(tmp, path)
    return name, time.time() - t0


def write_index():
    import numpy as np
    names = {}
    for spec in all_cases():
        name = case_name(*spec)
        p = os.path.join(OUT, name + ".npz")
        if not os.path.exists(p):
            continue
        d = np.load(p)
        names[name] = {"solver": spec[0], "wavelet": spec[1], "transfer": spec[2], "noise": spec[3],
                       "mu": d["mu"].tolist(), "iters": d["iters"].tolist(), "inner": d["inner"].tolist(),
                       "xnorm": float(d["xnorm"]), "rre_vs_phantom": float(d["rre"]),
                       "spread_x": float(d["spread_x"]), "spread_mu": d["spread_mu"].tolist(),
                       "spread_iters": d["spread_it"].tolist(),
                       "oracle_wall_s_one_thread": round(float(d["oracle_wall_s"]), 1)}
    meta = {"m": M, "psf": f"gaussian sigma={SIGMA} {PSF_SIZE}x{PSF_SIZE}", "levels": LEVELS, "seed": SEED,
            "phantom": f"{N_RECT} rectangles, {N_DISK} disks", "b": "A x_true + noise, rounded to float32",
            "samples": N_SAMPLES, "sample_seed": SAMPLE_SEED, "layout": "x_samples[j] = vec(X)[sample_index[j]], "
            "column-major", "perturbation": "float32 unit roundoff on every operator output, seeds "
            + ", ".join(map(str, PERTURB_SEEDS)), "cases": names}
    with open(os.path.join(OUT, "index.json"), "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--cases", default="", help="comma-separated case names (default: all)")
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import numpy as np
    os.makedirs(OUT, exist_ok=True)
    ip = os.path.join(OUT, "sample_index.npy")
    if not os.path.exists(ip):
        rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
        np.save(ip, np.sort(rng.choice(M * M, size=N_SAMPLES, replace=False)).astype(np.int64))
    want = set(a.cases.split(",")) if a.cases else None
    specs = [s for s in all_cases() if want is None or case_name(*s) in want]
    # one BLAS thread per worker; workers start by spawn (no inherited state)
    os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = "1"
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        for name, dt in pool.imap_unordered(run_case, specs):
            print(f"{name}: {dt:.0f} s", flush=True)
    write_index()


if __name__ == "__main__":
    main()
