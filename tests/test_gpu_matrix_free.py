"""The matrix-free stiffness of the structured Kuhn cube against the oracle.

amgh_kuhn_apply computes A x from the element coefficients alone (the
closed-form Kuhn element stiffness, pinned on the CPU in
test_oracle_assembly.py); it must equal the oracle's assembled product up to
rounding, with Dirichlet data on the whole boundary or on one face only, and
the mixed-precision solve with the matrix-free level-0 smoother must still
reach the oracle's control.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = {"grf9": lambda: W.cube_grf(N=9, features=64), "ball17": lambda: W.cube_ball(N=17, contrast=1e-3),
         "slabs33": lambda: W.cube_slabs(N=33)}


@pytest.mark.parametrize("name", list(CASES))
def test_matrix_free_apply_equals_assembled(name):
    import torch
    from paper_2001_11533_gb300 import amgh
    w = CASES[name]()
    prob = amgh.Problem.from_workload(w)
    orc = Oracle(w, setup=False)
    Kf = orc.scipy("Kfull")
    keep = np.flatnonzero(w.dirichlet == 0)
    A = Kf[keep][:, keep]
    x = np.random.default_rng(61).standard_normal(w.n_interior)
    ref = A @ x
    y = prob.kuhn_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= 1e-13
    y32 = prob.kuhn_apply(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    assert rel(y32.astype(np.float64), ref) <= 1e-5
    prob.close()


def test_matrix_free_rejects_other_meshes():
    from paper_2001_11533_gb300 import amgh
    import torch
    w = W.lshape_checkerboard(N=33)
    prob = amgh.Problem.from_workload(w)
    with pytest.raises(amgh.AmghError) as e:
        prob.kuhn_apply(torch.zeros(w.n_interior, dtype=torch.float64, device="cuda"))
    assert e.value.code == -1
    with pytest.raises(amgh.AmghError):
        prob.amg_setup(matrix_free=1)
    prob.close()


@pytest.mark.parametrize("name", ["grf9", "ball17"])
def test_matrix_free_smoother_solve_matches_oracle(name):
    from paper_2001_11533_gb300 import amgh
    w = CASES[name]()
    opts = dict(coarse_max=16, hessian_levels=2)
    prob = amgh.Problem.from_workload(w).amg_setup(precision=2, matrix_free=1, **opts)
    orc = Oracle(w, inner_tol=1e-13, mass_tol=1e-13, **opts)
    u, _, info = prob.solve(tol=1e-11, inner_tol=1e-12, mass_tol=1e-12, want_y=False)
    uo, _, io = orc.solve(precond=1, tol=1e-12)
    assert rel(u.cpu().numpy(), uo) <= 1e-8, (info, io)
