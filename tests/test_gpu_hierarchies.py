"""GPU parity of the alternative hierarchies and of the a_j diagnostics.

Aggressive first-level coarsening (Sec. 5.1) and the geometric hierarchy of
structured squares (Sec. 5.4) against the oracle: every level's matrices and
(for aggressive) the aggregates bit for bit, and converged controls.  The
power-method estimates of a~_j and a_j (Eq. aj-tilde, ajnumerical) against
the oracle's dense values, and the geometric rate a_j / a_j+1 near 1/4.
"""
import numpy as np
import pytest

from oracle.diagnostics import a_numbers
from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _same_hierarchy(prob, orc, aggregates=True):
    sz = orc.sizes()
    assert prob.sizes["state"] == sz["state"] and prob.sizes["control"] == sz["control"]
    for which, L in (("A", sz["Ls"]), ("My", sz["Ls"]), ("S", sz["Ls"] - 1), ("KN", sz["Lc"]),
                     ("Mu", sz["Lc"]), ("P", sz["Lc"] - 1), ("Myu", min(sz["Ls"], sz["Lc"]))):
        for l in range(L):
            for a, b in zip(prob.matrix(which, l)[:3], orc.matrix(which, l)[:3]):
                assert np.array_equal(a, b), (which, l)
    if aggregates:
        for hier, L in ((0, sz["Ls"]), (1, sz["Lc"])):
            for l in range(L - 1):
                ga, gn = prob.aggregates(hier, l)
                oa, on = orc.aggregates(hier, l)
                assert gn == on and np.array_equal(ga, oa), (hier, l)


@pytest.mark.parametrize("w", [W.lshape_checkerboard(N=65), W.cube_grf(N=9, features=64)],
                         ids=["lshape65", "cube9"])
def test_aggressive_hierarchy_bit_exact_and_solve(w):
    from paper_2001_11533_gb300 import amgh
    prob = amgh.Problem.from_workload(w).amg_setup(aggressive=1, coarse_max=16, hessian_levels=2)
    orc = Oracle(w, aggressive=1, coarse_max=16, hessian_levels=2, inner_tol=1e-13, mass_tol=1e-13)
    _same_hierarchy(prob, orc)
    u, _, info = prob.solve(tol=1e-12, inner_tol=1e-13, mass_tol=1e-13, want_y=False)
    uo, _, io = orc.solve(precond=1, tol=1e-12)
    assert rel(u.cpu().numpy(), uo) <= 1e-10, (info, io)


@pytest.mark.parametrize("N", [17, 65])
def test_geometric_hierarchy_bit_exact_and_two_grid_solve(N):
    from paper_2001_11533_gb300 import amgh
    w = W.unit_square(N, beta=1e-4, y_d="exact")
    prob = amgh.Problem.from_workload(w).amg_setup(geometric=1, coarse_max=1, hessian_levels=2, coarse_solve=2)
    orc = Oracle(w, geometric=1, coarse_max=1, hessian_levels=2, inner_tol=1e-13, mass_tol=1e-13)
    _same_hierarchy(prob, orc, aggregates=False)
    with pytest.raises(amgh.AmghError):
        prob.aggregates(0, 0)
    u, _, info = prob.solve(tol=1e-12, inner_tol=1e-13, mass_tol=1e-13, want_y=False)
    uo, _, io = orc.solve(precond=1, tol=1e-12)
    assert rel(u.cpu().numpy(), uo) <= 1e-10, (info, io)
    assert abs(info["outer_iters"] - io["outer_iters"]) <= 1


def test_geometric_rejects_other_meshes():
    from paper_2001_11533_gb300 import amgh
    for w in (W.lshape_checkerboard(N=33), W.cube_grf(N=9, features=16)):
        p = amgh.Problem.from_workload(w)
        with pytest.raises(amgh.AmghError) as e:
            p.amg_setup(geometric=1)
        assert e.value.code == -1
        p.close()


@pytest.mark.parametrize("kind", ["geometric", "amg", "aggressive"])
def test_aj_power_method_matches_dense(kind):
    """Power-method a~_j and a_j on the GPU against the oracle's dense norms: a
    lower bound within 1 % after 80 iterations, on every level pair."""
    from paper_2001_11533_gb300 import amgh
    w = W.unit_square(33)
    opts = {"geometric": dict(geometric=1, coarse_max=1), "amg": dict(coarse_max=8),
            "aggressive": dict(aggressive=1, coarse_max=8)}[kind]
    prob = amgh.Problem.from_workload(w).amg_setup(**opts)
    prob.set_solve_opts(inner_tol=1e-13, mass_tol=1e-13)
    orc = Oracle(w, **opts)
    L = min(prob.sizes["Ls"], prob.sizes["Lc"])
    rng = np.random.default_rng(41)
    for j in range(min(L - 1, 3)):
        a_ref, at_ref = a_numbers(orc, j)
        v0 = cuda(rng.standard_normal(prob.sizes["control"][j]))
        at = prob.aj_estimate(j, v0, weighted=False, iters=80)
        a = prob.aj_estimate(j, v0, weighted=True, iters=80)
        assert at_ref * 0.99 <= at <= at_ref * (1 + 1e-8), (j, at, at_ref)
        assert a_ref * 0.99 <= a <= a_ref * (1 + 1e-8), (j, a, a_ref)


def test_aj_geometric_rate_on_gpu():
    """Sec. 4 expects a_j <= C h_j^2 for geometric refinement: the GPU estimates
    on the 129^2 square give a_0 / a_1 close to 1/4."""
    from paper_2001_11533_gb300 import amgh
    w = W.unit_square(129)
    prob = amgh.Problem.from_workload(w).amg_setup(geometric=1, coarse_max=1)
    prob.set_solve_opts(inner_tol=1e-12, mass_tol=1e-12)
    v0 = cuda(np.random.default_rng(42).standard_normal(prob.sizes["n"]))
    a0 = prob.aj_estimate(0, v0, weighted=True, iters=60)
    v1 = cuda(np.random.default_rng(43).standard_normal(prob.sizes["control"][1]))
    a1 = prob.aj_estimate(1, v1, weighted=True, iters=60)
    assert 0.23 <= a0 / a1 <= 0.27, (a0, a1)


def test_experiment_tables_small():
    """The experiment drivers at small sizes: the Table 5 trend (geometric counts
    fall with N and stay at or below AMG's) and Table 7's (the multilevel
    preconditioner needs far fewer outer iterations than none)."""
    from paper_2001_11533_gb300 import experiments
    t5 = experiments.two_grid_table(sizes=(9, 17, 33), betas=(1e-4,))
    geo = [r["geometric_beta0.0001"] for r in t5["rows"]]
    amg = [r["amg_beta0.0001"] for r in t5["rows"]]
    assert all(isinstance(x, int) for x in geo + amg)
    assert geo[0] > geo[-1] and all(g <= a for g, a in zip(geo, amg))
    t7 = experiments.level_sweep_table(N=17, contrasts=(1e-2, 1.0), levels=(0, 2, 3))
    for row in t7["rows"]:
        none = row["none"]["outer"]
        assert row["2"]["outer"] * 3 < none, row
    t12 = experiments.a_numbers_table(N=33, levels=2, iters=40)
    geo = t12["rows"]["geometric"]
    assert 0.2 <= geo[1]["ratio_a_prev_over_a"] <= 0.32
    assert t12["rows"]["amg_aggressive"][0]["a"] > 2 * t12["rows"]["amg"][0]["a"]
