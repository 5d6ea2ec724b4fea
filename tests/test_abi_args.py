"""Argument checks of the C ABI that return before any device work, so they
run without a GPU: empty and out-of-range sizes, bad beta, null pointers,
invalid option values."""
import ctypes as C

import numpy as np
import pytest

from paper_2001_11533_gb300 import amgh


def _mesh(dim=2, nv=4, ne=2, dummy=None):
    arr = dummy if dummy is not None else np.zeros(16, dtype=np.float64)
    p = C.c_void_p(arr.ctypes.data)
    return amgh.amgh_mesh(dim, nv, p, ne, p, p, 0)


def _create(mesh, beta=1.0):
    kappa = np.ones(8)
    yd = np.zeros(8)
    h = C.c_void_p()
    st = amgh.lib().amgh_problem_create(C.byref(mesh), C.c_void_p(kappa.ctypes.data), C.c_double(beta),
                                        C.c_void_p(yd.ctypes.data), 0, C.byref(h))
    return st, h


@pytest.mark.parametrize("kw,beta", [
    (dict(ne=0), 1.0),                  # no elements
    (dict(nv=0), 1.0),                  # no vertices
    (dict(dim=1), 1.0),                 # unsupported dimension
    (dict(dim=4), 1.0),
    (dict(nv=2 ** 31), 1.0),            # more vertices than int32 indices address
    (dict(ne=2 ** 30), 1.0),            # n_elements * (dim + 1) >= 2^31
    (dict(), 0.0),                      # beta must be > 0
    (dict(), -1.0),
    (dict(), float("inf")),
    (dict(), float("nan")),
])
def test_create_rejects(kw, beta):
    dummy = np.zeros(16)
    st, h = _create(_mesh(dummy=dummy, **kw), beta)
    assert st == -1 and not h.value


def test_null_arguments():
    L = amgh.lib()
    h = C.c_void_p()
    assert L.amgh_problem_create(None, None, C.c_double(1.0), None, 0, C.byref(h)) == -1
    assert L.amgh_amg_setup(None, None) == -1
    assert L.amgh_solve(None, None, None, None, None, None) == -1
    assert L.amgh_hessian_apply(None, None, None, 1) == -1
    assert L.amgh_hessian_apply(None, None, None, 4) == -1
    assert L.amgh_precond_apply(None, None, None, 4) == -1
    assert L.amgh_solve_block(None, None, 3, None, None, None) == -1
    assert L.amgh_batch_set_block(None, 1) == -1
    assert L.amgh_batch_create(None, 0, C.byref(h)) == -1
    assert L.amgh_problem_share(None, C.byref(h)) == -1
    assert L.amgh_aggregate_noalloc(0, None, None, None, 0.08, None, None, None) == -1
    assert L.amgh_aggregate_noalloc(40000, None, None, None, 0.08, None, None, None) == -1
    L.amgh_problem_destroy(None)
    L.amgh_batch_destroy(None)


def test_defaults_and_status_strings():
    o = amgh.amg_opts()
    assert (o.max_levels, o.theta, o.coarse_max, o.smooth_degree, o.precision) == (25, 0.08, 256, 2, 0)
    assert (o.coarse_solve, o.fuse_coarse, o.autotune) == (0, 0, 0)
    so = amgh.solve_opts()
    assert (so.tol, so.max_iter, so.coarse_tol, so.level_fallback) == (1e-8, 200, 1e-4, 0)
    for code in range(0, -9, -1):
        assert amgh.lib().amgh_status_string(code)
    with pytest.raises(TypeError):
        amgh.amg_opts(no_such_field=1)


def test_dense_probe_and_debug_entry_points_reject_bad_arguments():
    """The dense inverse, the FP64 rate probe and the grid-barrier test hook check
    their arguments before touching the device (n in 1..4096, non-null buffers,
    kind 0 or 1, a poll limit of -1 or more)."""
    L = amgh.lib()
    buf = np.zeros(4, dtype=np.float64)
    p = C.c_void_p(buf.ctypes.data)
    info = C.c_int32(7)
    for n, a, inv in [(0, p, p), (-3, p, p), (4097, p, p), (2, None, p), (2, p, None)]:
        info.value = 7
        assert L.amgh_dense_spd_inverse(n, a, inv, None, C.byref(info)) == -1
        assert info.value == 0  # info is cleared even when the call is refused
    assert L.amgh_dense_spd_inverse(0, p, p, None, None) == -1
    t = C.c_double(5.0)
    assert L.amgh_fp64_peak(2, None, C.byref(t)) == -1
    assert L.amgh_fp64_peak(-1, None, C.byref(t)) == -1
    assert L.amgh_fp64_peak(0, None, None) == -1
    assert L.amgh_debug_grid_polls(-2) == -1
