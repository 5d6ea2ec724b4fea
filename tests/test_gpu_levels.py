"""Coarsest Hessian level by plain CG (Sec. 5.2) and the fallback to fewer
Hessian levels when the multilevel preconditioner is indefinite (Sec. 3.2;
the paper cuts levels for this reason in Sec. 5.5-5.6): the CUDA path through
the C ABI against the FP64 oracle with the same levels."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(inner_tol=1e-13, mass_tol=1e-13)


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(w, **amg):
    from paper_2001_11533_gb300 import amgh
    return amgh.Problem.from_workload(w).amg_setup(**amg)


def test_coarse_cg_matches_oracle():
    w = W.lshape_checkerboard(N=65)
    prob = _problem(w, coarse_max=32, coarse_solve=1)
    u, _, info = prob.solve(tol=1e-12, coarse_tol=1e-4, **TIGHT)
    assert info["coarse_iters"] > 0 and info["fallbacks"] == 0
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    orc.set_coarse_solve(1, tol=1e-4)
    uo, _, io = orc.solve(precond=1, tol=1e-12)
    assert rel(u.cpu().numpy(), uo) <= 1e-10
    # the preconditioner only changes the iteration, not the answer
    assert abs(info["outer_iters"] - io["outer_iters"]) <= 1


def test_coarse_cg_single_apply_matches_oracle():
    w = W.lshape_checkerboard(N=65)
    prob = _problem(w, coarse_max=32, coarse_solve=1)
    prob.set_solve_opts(coarse_tol=1e-4, **TIGHT)
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    orc.set_coarse_solve(1, tol=1e-4)
    r = np.random.default_rng(11).standard_normal(w.n_vertices)
    z = prob.precond_apply(cuda(r)).cpu().numpy()
    zo = orc.precond(r)
    # same CG steps on both sides; the iterates differ by rounding of the
    # inner solves (1e-13) amplified by the coarse CG
    assert rel(z, zo) <= 1e-8


@pytest.mark.parametrize("coarse_solve", [0, 1])
def test_level_fallback_matches_oracle_with_fewer_levels(coarse_solve):
    # beta = 1.1e-4 on a 65^2 square with 4 Hessian levels: indefinite W
    w = W.batch_squares(sizes=(65,), per_size=3, rhs=1)[2]
    prob = _problem(w, coarse_max=32, coarse_solve=coarse_solve)
    ell0 = prob.query_sizes()["ell"]
    _, _, bad = prob.solve(tol=1e-12, raise_on_error=False, **TIGHT)
    assert bad["status"] == -6            # INDEFINITE without the fallback
    prob = _problem(w, coarse_max=32, coarse_solve=coarse_solve)
    u, _, info = prob.solve(tol=1e-12, level_fallback=1, **TIGHT)
    assert info["fallbacks"] >= 1
    assert info["hessian_levels"] == ell0 - info["fallbacks"] >= 2
    orc = Oracle(w, coarse_max=32, hessian_levels=info["hessian_levels"], inner_tol=1e-13,
                 mass_tol=1e-13)
    if coarse_solve:
        orc.set_coarse_solve(1, tol=1e-4)
    uo, _, _ = orc.solve(precond=1, tol=1e-12)
    assert rel(u.cpu().numpy(), uo) <= 1e-10
    # the reduction persists for the next solve of this problem
    _, _, again = prob.solve(tol=1e-10, level_fallback=1)
    assert again["fallbacks"] == 0 and again["hessian_levels"] == info["hessian_levels"]
