#!/usr/bin/env python
"""Writes the FP64 oracle's result for one case of the large-image workload
into tests/golden/m2048_oracle/ (<case>.npz plus index.json).

Workload: a 2048 x 2048 piecewise-constant phantom (80 rectangles, 40 disks,
seed 0), Gaussian PSF sigma = 6 on 31 x 31 (sum 1), b = A x_true + e with e
at 1 % of ||A x_true|| (Sec. 5), rounded to bfloat16 (the storage precision
of the GPU path, which then sees exactly the same input); a 5-level
Daubechies-4 V-cycle (Alg. 4) of the given solver and transfer strategy
(Alg. 1-3), gamma by GCV on every level (Sec. 3).

Stored: gamma per level, outer and LSQR iteration counts per level, ||x||,
x at 16384 fixed pixels (seed 2048), the error against the phantom and the
wall time of the solve. With --rerun SEED the same solve runs under the
bfloat16 rounding-noise model of tests/perturb.py (bfloat16 unit roundoff on
the LSQR operator outputs and the per-pixel planes, float32 inside GCV) and
is stored beside it as <case>.rerun<SEED>.npz: the oracle's own spread under
the storage precision of the GPU path. One solve takes about 1.5 h.

This script calls only oracle/, the input generator and that noise model.

    python tests/golden/make_m2048_oracle.py mm X
    python tests/golden/make_m2048_oracle.py mm X --rerun 12345
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "m2048_oracle")
M, SIGMA, PSF_SIZE, LEVELS, SEED, NOISE = 2048, 6.0, 31, 5, 0, 0.01
N_SAMPLES, SAMPLE_SEED = 16384, 2048


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even) through float32."""
    import numpy as np
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def main():
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import operators as O
    from oracle import solvers as S
    from paper_2608_17123_b300 import inputs as I
    solver, transfer = sys.argv[1], sys.argv[2]
    rerun = int(sys.argv[4]) if len(sys.argv) > 4 and sys.argv[3] == "--rerun" else None
    name = f"gauss31-{solver}-db4-{transfer}"
    os.makedirs(OUT, exist_ok=True)
    ip = os.path.join(OUT, "sample_index.npy")
    if not os.path.exists(ip):
        rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
        np.save(ip, np.sort(rng.choice(M * M, size=N_SAMPLES, replace=False)).astype(np.int64))
    idx = np.load(ip)
    g = I.gaussian_factor(SIGMA, PSF_SIZE)
    A = O.KronOp.from_factors(M, g, g)
    R = int(round(40 * math.sqrt(M / 512)))
    x_true = I.phantom(M, R, R // 2, SEED)
    b = to_bf16(I.add_noise(A.apply(x_true), I.noise_direction(M, 10_000 + SEED), NOISE))
    t0 = time.time()
    if rerun is not None:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from perturb import noisy
        r = noisy(lambda: S.mgm(b, A, solver, "db4", LEVELS, transfer), "bf16", rerun)
        wall = time.time() - t0
        x = r["x"]
        np.savez(os.path.join(OUT, f"{name}.rerun{rerun}.npz"), x_samples=x.T.reshape(-1)[idx].astype(np.float32),
                 mu=np.array(r["mu"]), iters=np.array(r["iters"], dtype=np.int32),
                 inner=np.array(r["inner"], dtype=np.int32), oracle_wall_s=np.float64(wall))
        print(name, "rerun", rerun, f"{wall:.0f} s", r["iters"], r["mu"], flush=True)
        return
    r = S.mgm(b, A, solver, "db4", LEVELS, transfer)
    wall = time.time() - t0
    x = r["x"]
    np.savez(os.path.join(OUT, name + ".npz"), x_samples=x.T.reshape(-1)[idx].astype(np.float32),
             mu=np.array(r["mu"]), iters=np.array(r["iters"], dtype=np.int32),
             inner=np.array(r["inner"], dtype=np.int32), xnorm=np.float64(np.linalg.norm(x)),
             rre=np.float64(np.linalg.norm(x - x_true) / np.linalg.norm(x_true)), oracle_wall_s=np.float64(wall))
    ipath = os.path.join(OUT, "index.json")
    meta = json.load(open(ipath)) if os.path.exists(ipath) else {
        "m": M, "psf": f"gaussian sigma={SIGMA} {PSF_SIZE}x{PSF_SIZE}", "levels": LEVELS, "wavelet": "db4",
        "seed": SEED, "noise": NOISE, "phantom": f"{R} rectangles, {R // 2} disks",
        "b": "A x_true + noise, rounded to bfloat16", "samples": N_SAMPLES, "sample_seed": SAMPLE_SEED,
        "layout": "x_samples[j] = vec(X)[sample_index[j]], column-major", "cases": {}}
    meta["cases"][name] = {"solver": solver, "transfer": transfer, "mu": list(map(float, r["mu"])),
                           "iters": list(map(int, r["iters"])), "inner": list(map(int, r["inner"])),
                           "xnorm": float(np.linalg.norm(x)),
                           "rre_vs_phantom": float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true)),
                           "oracle_wall_s": round(wall, 1)}
    with open(ipath, "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)
    print(name, f"{wall:.0f} s", r["iters"], r["mu"], flush=True)


if __name__ == "__main__":
    main()
