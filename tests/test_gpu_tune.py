"""Layout autotuning at setup: whatever layout each operator gets, the
solve still matches the FP64 oracle, and a second setup of the same mesh
reuses the remembered choices (same bits)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_autotuned_solve_matches_oracle():
    from paper_2001_11533_gb300 import amgh
    w = W.lshape_checkerboard(N=129)
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    uo, _, _ = orc.solve(precond=1, tol=1e-12)
    runs = []
    for k in range(2):
        p = amgh.Problem.from_workload(w).amg_setup(coarse_max=32, autotune=1)
        u, _, info = p.solve(tol=1e-12, inner_tol=1e-13, mass_tol=1e-13)
        assert rel(u.cpu().numpy(), uo) <= 1e-10
        runs.append(u.cpu().numpy())
    assert np.array_equal(runs[0], runs[1])
    pm = amgh.Problem.from_workload(w).amg_setup(coarse_max=32, autotune=1, precision=2)
    um, _, _ = pm.solve(tol=1e-11, inner_tol=1e-12, mass_tol=1e-12)
    assert rel(um.cpu().numpy(), uo) <= 1e-8
