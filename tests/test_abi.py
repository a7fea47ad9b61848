"""The C-ABI library builds, loads and exports every entry point that
include/deblur.h declares (no GPU needed: nothing is launched)."""
import ctypes
import os
import subprocess

from paper_2608_17123_b300 import _lib


def test_library_exports_header_symbols():
    L = _lib.lib()
    names = _lib.header_symbols()
    assert "deblur_solve" in names and "db_context_create" in names
    for n in names:
        assert hasattr(L, n), n
    # symbols are exported with C linkage
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in names:
        assert n in exported, n


def test_defaults_and_footprint():
    o, g = _lib.default_opts()
    assert (o.tol_fine, o.tol_coarse, o.kmax, o.lsqr_maxit) == (1e-3, 1e-6, 50, 100)
    assert (o.eps_irls, o.eps_mm, o.tau_sb) == (0.03, 0.03, 0.005)
    assert (g.grid_points, g.gcv_estimates, g.proj_dim, g.proj_dim_max) == (50, 3, 40, 160)
    L = _lib.lib()
    f512 = L.db_footprint_bytes(512, 3, 15, 1, ctypes.byref(g))
    f1k = L.db_footprint_bytes(1024, 3, 15, 1, ctypes.byref(g))
    assert f1k > 3 * f512 > 0


def test_invalid_arguments_rejected_without_gpu_work():
    L = _lib.lib()
    # null / bad sizes are rejected before any launch
    assert L.db_apply_L(0, None, None, 1, None) == 1
    assert L.db_restrict(6, 0, None, None, 1, None) == 1
    assert L.deblur_solve(None, None, 64, None, 9, 0, 0, 2, 1, None, None, None, None, None, None, 0, None) == 1
