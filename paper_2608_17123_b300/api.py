"""Python front end of libdeblur: same names as the C-ABI, argument
marshalling only.

Images passed as numpy arrays are m x m arrays indexed [r, c]; they are
handed to the library as column-major float64 buffers. Device entry points
take torch CUDA tensors that already hold column-major buffers (use
``inputs.to_colmajor`` before uploading).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .inputs import to_colmajor, from_colmajor


def _ptr(t):
    """Raw device pointer of a torch tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        try:
            import torch
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return C.c_void_p(0)
    return C.c_void_p(int(stream))


class Context:
    """A libdeblur context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.handle = C.c_void_p()
        L.check(L.lib().db_context_create(C.byref(self.handle), device, hbm_budget_bytes))

    def set_profiling(self, on=True):
        L.check(L.lib().db_set_profiling(self.handle, int(on)), self.handle)

    def set_autotune(self, on=True):
        L.check(L.lib().db_set_autotune(self.handle, int(on)), self.handle)

    def stats(self):
        st = L.DbStats()
        L.check(L.lib().db_get_stats(self.handle, C.byref(st)), self.handle)
        return {k: getattr(st, k) for k, _ in L.DbStats._fields_}

    def reset_stats(self):
        L.check(L.lib().db_reset_stats(self.handle), self.handle)

    def close(self):
        if self.handle:
            L.lib().db_context_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = None


def default_context():
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(0)
    return _default_ctx


def make_opts(precision="fp32", **kw):
    o, g = L.default_opts()
    o.precision = L.PRECISIONS[precision]
    for k, v in kw.items():
        if hasattr(o, k) and k != "precision":
            setattr(o, k, v)
        elif hasattr(g, k):
            setattr(g, k, v)
        else:
            raise KeyError(k)
    return o, g


def deblur_solve(b, psf, solver="irls", wavelet="haar", levels=2, transfer="X", precision="fp32",
                 ctx=None, stream=None, **options):
    """One V-cycle solve (Alg. 4) on host arrays. Returns dict(x, mu, iters, inner)."""
    ctx = ctx or default_context()
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    psf = np.asarray(psf, dtype=np.float64)
    S = psf.shape[0]
    o, g = make_opts(precision, **options)
    bb = to_colmajor(b)
    pp = to_colmajor(psf)
    x = np.empty(m * m, dtype=np.float64)
    mu = np.zeros(levels, dtype=np.float64)
    it = np.zeros(levels, dtype=np.int32)
    inner = np.zeros(levels, dtype=np.int32)
    st = L.lib().deblur_solve(ctx.handle, bb.ctypes.data, m, pp.ctypes.data, S, L.SOLVERS[solver],
                              L.WAVELETS[wavelet], levels, L.TRANSFERS[transfer], C.byref(g), C.byref(o),
                              x.ctypes.data, mu.ctypes.data, it.ctypes.data, inner.ctypes.data, 0,
                              _stream(stream))
    L.check(st, ctx.handle)
    return dict(x=from_colmajor(x, m), mu=list(mu), iters=[int(v) for v in it], inner=[int(v) for v in inner])


def deblur_solve_batch(problems, precision="fp32", ctx=None, stream=None, **options):
    """Batched solves. ``problems``: list of dicts with keys b (m x m array),
    psf, solver, wavelet, levels, transfer. Returns a list of result dicts."""
    ctx = ctx or default_context()
    o, g = make_opts(precision, **options)
    keep, reqs, outs = [], (L.DbRequest * len(problems))(), []
    for i, pr in enumerate(problems):
        b = np.asarray(pr["b"], dtype=np.float64)
        m = b.shape[0]
        psf = np.asarray(pr["psf"], dtype=np.float64)
        lv = pr.get("levels", 2)
        bb, pp = to_colmajor(b), to_colmajor(psf)
        x = np.empty(m * m)
        mu = np.zeros(lv)
        it = np.zeros(lv, dtype=np.int32)
        inner = np.zeros(lv, dtype=np.int32)
        keep += [bb, pp, x, mu, it, inner]
        r = reqs[i]
        r.b, r.m, r.psf, r.psf_size = bb.ctypes.data, m, pp.ctypes.data, psf.shape[0]
        r.solver = L.SOLVERS[pr.get("solver", "irls")]
        r.wavelet = L.WAVELETS[pr.get("wavelet", "haar")]
        r.levels = lv
        r.transfer = L.TRANSFERS[pr.get("transfer", "X")]
        r.x, r.mu_per_level, r.iters_per_level, r.inner_iters_per_level = (
            x.ctypes.data, mu.ctypes.data, it.ctypes.data, inner.ctypes.data)
        outs.append((m, x, mu, it, inner))
    L.check(L.lib().deblur_solve_batch(ctx.handle, len(problems), reqs, C.byref(g), C.byref(o), 0,
                                       _stream(stream)), ctx.handle)
    return [dict(x=from_colmajor(x, m), mu=list(mu), iters=[int(v) for v in it], inner=[int(v) for v in inner])
            for (m, x, mu, it, inner) in outs]


def deblur_solve_batch_device(problems, precision="fp32", ctx=None, stream=None, **options):
    """Batched solves on device buffers. ``problems``: list of dicts with keys
    b, psf, x (torch float64 CUDA tensors, column-major), m, psf_size, solver,
    wavelet, levels, transfer. Returns per problem dict(mu, iters, inner)."""
    ctx = ctx or default_context()
    o, g = make_opts(precision, **options)
    reqs, outs = (L.DbRequest * len(problems))(), []
    for i, pr in enumerate(problems):
        lv = pr.get("levels", 2)
        mu = np.zeros(lv)
        it = np.zeros(lv, dtype=np.int32)
        inner = np.zeros(lv, dtype=np.int32)
        r = reqs[i]
        r.b, r.m, r.psf, r.psf_size = pr["b"].data_ptr(), pr["m"], pr["psf"].data_ptr(), pr["psf_size"]
        r.solver = L.SOLVERS[pr.get("solver", "irls")]
        r.wavelet = L.WAVELETS[pr.get("wavelet", "haar")]
        r.levels = lv
        r.transfer = L.TRANSFERS[pr.get("transfer", "X")]
        r.x, r.mu_per_level, r.iters_per_level, r.inner_iters_per_level = (
            pr["x"].data_ptr(), mu.ctypes.data, it.ctypes.data, inner.ctypes.data)
        outs.append((mu, it, inner))
    L.check(L.lib().deblur_solve_batch(ctx.handle, len(problems), reqs, C.byref(g), C.byref(o), 1,
                                       _stream(stream)), ctx.handle)
    return [dict(mu=list(mu), iters=[int(v) for v in it], inner=[int(v) for v in inner]) for (mu, it, inner) in outs]


def deblur_solve_device(b_dev, psf_dev, m, S, x_dev, solver="irls", wavelet="haar", levels=2, transfer="X",
                        precision="fp32", ctx=None, stream=None, **options):
    """Same call on device buffers (torch float64 CUDA tensors, column-major)."""
    ctx = ctx or default_context()
    o, g = make_opts(precision, **options)
    mu = np.zeros(levels, dtype=np.float64)
    it = np.zeros(levels, dtype=np.int32)
    inner = np.zeros(levels, dtype=np.int32)
    st = L.lib().deblur_solve(ctx.handle, _ptr(b_dev), m, _ptr(psf_dev), S, L.SOLVERS[solver],
                              L.WAVELETS[wavelet], levels, L.TRANSFERS[transfer], C.byref(g), C.byref(o),
                              _ptr(x_dev), mu.ctypes.data, it.ctypes.data, inner.ctypes.data, 1, _stream(stream))
    L.check(st, ctx.handle)
    return dict(mu=list(mu), iters=[int(v) for v in it], inner=[int(v) for v in inner])


# ---- operator-level calls (torch CUDA tensors, column-major) -----------------

def _prec(t):
    import torch
    return {torch.float64: 0, torch.float32: 1}[t.dtype]


def apply_blur(psf, m, x, y, level=0, wavelet="haar", transpose=False, ctx=None, stream=None):
    ctx = ctx or default_context()
    pp = to_colmajor(np.asarray(psf, dtype=np.float64))
    L.check(L.lib().db_apply_blur(ctx.handle, pp.ctypes.data, pp.shape[0], m, L.WAVELETS[wavelet], level,
                                  int(transpose), _ptr(x), _ptr(y), _prec(x), _stream(stream)), ctx.handle)


def sumsq(x, stream=None):
    """sum(x^2) of a torch CUDA tensor (float64, float32 or bfloat16) by the
    library's LSQR-norm reduction (db_sumsq)."""
    import torch
    prec = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}[x.dtype]
    out = C.c_double(0.0)
    L.check(L.lib().db_sumsq(_ptr(x), x.numel(), prec, C.byref(out), _stream(stream)))
    return out.value


def apply_L(m, x, q, stream=None):
    L.check(L.lib().db_apply_L(m, _ptr(x), _ptr(q), _prec(x), _stream(stream)))


def apply_Lt(m, q, x, stream=None):
    L.check(L.lib().db_apply_Lt(m, _ptr(q), _ptr(x), _prec(x), _stream(stream)))


def restrict(m, x, y, wavelet="haar", stream=None):
    L.check(L.lib().db_restrict(m, L.WAVELETS[wavelet], _ptr(x), _ptr(y), _prec(x), _stream(stream)))


def prolong(mc, y, x, wavelet="haar", stream=None):
    L.check(L.lib().db_prolong(mc, L.WAVELETS[wavelet], _ptr(y), _ptr(x), _prec(x), _stream(stream)))


def aux_prolong(mc, qc, qf, wavelet="haar", stream=None):
    L.check(L.lib().db_aux_prolong(mc, L.WAVELETS[wavelet], _ptr(qc), _ptr(qf), _prec(qc), _stream(stream)))


def lsqr_solve(psf, m, solver, gamma, b, x0, aux0, aux1, x_out, ctx=None, stream=None, **options):
    ctx = ctx or default_context()
    pp = to_colmajor(np.asarray(psf, dtype=np.float64))
    o, _ = make_opts("fp64" if _prec(b) == 0 else "fp32", **options)
    its = C.c_int(0)
    L.check(L.lib().db_lsqr_solve(ctx.handle, pp.ctypes.data, pp.shape[0], m, L.SOLVERS[solver], gamma,
                                  _ptr(b), _ptr(x0), _ptr(aux0), _ptr(aux1), _ptr(x_out), C.byref(o),
                                  C.byref(its), _prec(b), _stream(stream)), ctx.handle)
    return its.value


def lsqr_solve_static(psf, m, solver, gamma, b, x0, aux0, aux1, x_out, stream=None, **options):
    """db_lsqr_solve_static: lsqr_solve without a context or any device
    allocation (static 16 MiB workspace; m <= 256, PSF <= 31 x 31)."""
    pp = to_colmajor(np.asarray(psf, dtype=np.float64))
    o, _ = make_opts("fp64" if _prec(b) == 0 else "fp32", **options)
    its = C.c_int(0)
    L.check(L.lib().db_lsqr_solve_static(pp.ctypes.data, pp.shape[0], m, L.SOLVERS[solver], gamma,
                                         _ptr(b), _ptr(x0), _ptr(aux0), _ptr(aux1), _ptr(x_out), C.byref(o),
                                         C.byref(its), _prec(b), _stream(stream)))
    return its.value


def gcv_select(psf, m, solver, b, aux0=None, aux1=None, ctx=None, stream=None, **options):
    ctx = ctx or default_context()
    pp = to_colmajor(np.asarray(psf, dtype=np.float64))
    _, g = make_opts("fp32", **options)
    gamma = C.c_double(0.0)
    L.check(L.lib().db_gcv_select(ctx.handle, pp.ctypes.data, pp.shape[0], m, L.SOLVERS[solver], _ptr(b),
                                  _ptr(aux0), _ptr(aux1), C.byref(g), C.byref(gamma), _prec(b),
                                  _stream(stream)), ctx.handle)
    return gamma.value


class Server:
    """Continuous-batching solver (db_server_*): submit() returns a ticket at
    once; poll() waits for it and returns (result dict, latency in ms)."""

    def __init__(self, max_resident=8, max_m=1024, hbm_budget_bytes=0, ctx=None, **options):
        self.ctx = ctx or Context(0)
        o, g = make_opts("fp32", **options)
        so = L.DbServerOpts()
        so.max_resident, so.max_m, so.hbm_budget_bytes = max_resident, max_m, hbm_budget_bytes
        so.opts, so.gcv = o, g
        self.handle = C.c_void_p()
        L.check(L.lib().db_server_create(self.ctx.handle, C.byref(so), C.byref(self.handle)), self.ctx.handle)
        self._live = {}

    def submit(self, b, psf, solver="irls", wavelet="haar", levels=2, transfer="X"):
        b = np.asarray(b, dtype=np.float64)
        m = b.shape[0]
        psf = np.asarray(psf, dtype=np.float64)
        bb, pp = to_colmajor(b), to_colmajor(psf)
        x = np.empty(m * m)
        mu = np.zeros(levels)
        it = np.zeros(levels, dtype=np.int32)
        inner = np.zeros(levels, dtype=np.int32)
        r = L.DbRequest()
        r.b, r.m, r.psf, r.psf_size = bb.ctypes.data, m, pp.ctypes.data, psf.shape[0]
        r.solver, r.wavelet, r.levels = L.SOLVERS[solver], L.WAVELETS[wavelet], levels
        r.transfer = L.TRANSFERS[transfer]
        r.x, r.mu_per_level, r.iters_per_level, r.inner_iters_per_level = (
            x.ctypes.data, mu.ctypes.data, it.ctypes.data, inner.ctypes.data)
        t = C.c_uint64(0)
        L.check(L.lib().db_server_submit(self.handle, C.byref(r), C.byref(t)), self.ctx.handle)
        self._live[t.value] = (m, x, mu, it, inner, bb, pp, r)
        return t.value

    def poll(self, ticket, timeout_us=-1):
        lat = C.c_double(0.0)
        st = L.lib().db_server_poll(self.handle, ticket, timeout_us, C.byref(lat))
        if st == 4:  # DB_ETIMEOUT
            return None
        if st != 0:
            self._live.pop(ticket, None)
        L.check(st, self.ctx.handle)
        m, x, mu, it, inner, _, _, _ = self._live.pop(ticket)
        return dict(x=from_colmajor(x, m), mu=list(mu), iters=[int(v) for v in it],
                    inner=[int(v) for v in inner]), lat.value

    def cancel(self, ticket):
        L.check(L.lib().db_server_cancel(self.handle, ticket), self.ctx.handle)

    def close(self):
        if self.handle:
            L.lib().db_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
