"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/amgh.h (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "amgh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amgh_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_11533_gb300 import _build
    return _build.build()


def test_every_declared_symbol_exported(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(libpath):
    from paper_2001_11533_gb300 import amgh
    assert amgh.declared_symbols() == _declared()


def test_status_strings(libpath):
    from paper_2001_11533_gb300 import amgh
    L = amgh.lib()
    assert L.amgh_status_string(0) == b"ok"
    assert L.amgh_status_string(-6).startswith(b"indefinite")


def test_defaults_without_gpu(libpath):
    from paper_2001_11533_gb300 import amgh
    o = amgh.amg_opts()
    assert (o.max_levels, o.coarse_max, o.smooth_degree, o.theta) == (25, 256, 2, 0.08)
    s = amgh.solve_opts()
    assert (s.tol, s.inner_tol, s.precond) == (1e-8, 1e-10, 1)


def test_stacked_vectors_are_column_major():
    """A (k, n) contiguous tensor is k columns of n, i.e. the column-major
    n x k block the C ABI expects; other layouts are refused."""
    import torch
    from paper_2001_11533_gb300 import amgh
    cols = amgh.Problem._cols
    assert cols(torch.zeros(7, dtype=torch.float64)) == 1
    assert cols(torch.zeros(3, 7, dtype=torch.float64)) == 3
    with pytest.raises(ValueError):
        cols(torch.zeros(7, 3, dtype=torch.float64).t())
