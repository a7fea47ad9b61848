"""Failure detection without a GPU fault: every device wait is bounded and
ends in a status the host reads; host-side failures (allocation beyond the
budget, withdrawn or unfinished requests) come back as statuses too. After
each failure the same context solves correctly.

* A device wait that runs out: the persistent LSQR launch is given a wait
  limit of zero (barrier_timeout_us = 0), so its first grid-barrier wait
  expires; every block leaves the launch and the call returns DB_ETIMEOUT.
* Allocation failure: a context whose HBM budget is below the workspace of
  the solve returns DB_ENOMEM before allocating.
* A ticket polled with no wait while it is queued behind an occupied slot
  returns DB_ETIMEOUT; a withdrawn request returns DB_ECANCELLED.
"""
import numpy as np
import pytest

from oracle import operators as O
from paper_2608_17123_b300 import api
from paper_2608_17123_b300 import inputs as I
from paper_2608_17123_b300._lib import DeblurError

from helpers import img_to_dev, rel

pytestmark = pytest.mark.gpu
DB_ENOMEM, DB_ETIMEOUT, DB_ECANCELLED = 2, 4, 6


def make(m, sigma=2.0, Sz=9, seed=0):
    x_true = I.phantom(m, 8, 4, seed)
    g = I.gaussian_factor(sigma, Sz)
    A = O.KronOp.from_factors(m, g, g)
    return I.add_noise(A.apply(x_true), I.noise_direction(m, 700 + seed), 0.01), np.outer(g, g)


@pytest.mark.parametrize("m", [64, 512])
def test_barrier_wait_limit_returns_timeout_and_context_recovers(m):
    b, psf = make(m)
    ctx = api.Context(0)
    try:
        with pytest.raises(DeblurError) as e:
            api.deblur_solve(b, psf, "mm", "haar", 2, "X", precision="fp32", ctx=ctx, barrier_timeout_us=0)
        assert e.value.status == DB_ETIMEOUT
        r = api.deblur_solve(b, psf, "mm", "haar", 2, "X", precision="fp32", ctx=ctx)
    finally:
        ctx.close()
    fresh = api.Context(0)
    try:
        r2 = api.deblur_solve(b, psf, "mm", "haar", 2, "X", precision="fp32", ctx=fresh)
    finally:
        fresh.close()
    assert r["iters"] == r2["iters"] and rel(r["x"], r2["x"]) == 0.0


def test_lsqr_wait_limit_returns_timeout():
    import torch
    m = 256
    b, psf = make(m)
    bd = img_to_dev(b, torch.float32)
    xo = torch.empty(m * m, device="cuda", dtype=torch.float32)
    ctx = api.Context(0)
    try:
        with pytest.raises(DeblurError) as e:
            api.lsqr_solve(psf, m, "mm", 1e-3, bd, None, None, None, xo, ctx=ctx, barrier_timeout_us=0)
        assert e.value.status == DB_ETIMEOUT
        its = api.lsqr_solve(psf, m, "mm", 1e-3, bd, None, None, None, xo, ctx=ctx)
        assert its >= 1 and bool(torch.isfinite(xo).all())
    finally:
        ctx.close()


def test_budget_below_workspace_is_enomem():
    b, psf = make(64)
    small = api.Context(0, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(DeblurError) as e:
            api.deblur_solve(b, psf, "irls", "haar", 2, "X", ctx=small)
        assert e.value.status == DB_ENOMEM
    finally:
        small.close()
    ok = api.Context(0)
    try:
        r = api.deblur_solve(b, psf, "irls", "haar", 2, "X", ctx=ok)
        assert r["iters"][0] >= 1
    finally:
        ok.close()


def test_server_poll_timeout_and_cancel():
    srv = api.Server(max_resident=1, max_m=128, ctx=api.Context(0))
    try:
        b0, p0 = make(128, seed=1)
        b1, p1 = make(64, seed=2)
        b2, p2 = make(64, seed=3)
        t0 = srv.submit(b0, p0, "irls", "db4", 3, "X")
        t1 = srv.submit(b1, p1, "mm", "haar", 2, "D")
        t2 = srv.submit(b2, p2, "sb", "haar", 2, "X")
        # t1 waits behind t0 in the single slot: not done after a zero wait
        assert srv.poll(t1, timeout_us=0) is None
        srv.cancel(t2)                      # still queued: leaves at once
        with pytest.raises(DeblurError) as e:
            srv.poll(t2)
        assert e.value.status == DB_ECANCELLED
        srv.cancel(t0)                      # resident (or queued): retired at a step boundary
        with pytest.raises(DeblurError) as e:
            srv.poll(t0)
        assert e.value.status == DB_ECANCELLED
        r1, lat = srv.poll(t1)
        assert lat > 0.0
    finally:
        srv.close()
    alone = api.deblur_solve(b1, p1, "mm", "haar", 2, "D", precision="fp32")
    assert r1["iters"] == alone["iters"] and rel(r1["x"], alone["x"]) <= 1e-12
