"""Pins for the oracle's alternative hierarchies and the a_j diagnostics.

Geometric hierarchy (the comparison of Sec. 5.4): nested structured square
grids with P1 interpolation.  Checked against linear-function reproduction
and against a direct assembly on the coarse grid (for nested P1 spaces the
Galerkin product is the rediscretised matrix), and by the rate of the
two-level approximation numbers: Sec. 4 expects a_j <= C h_j^2, i.e. a ratio
a_j / a_j+1 near 1/4 for geometric refinement (Tables 1-2).

Aggressive first-level coarsening (Sec. 5.1, reading for smoothed
aggregation: the level-0 aggregates are aggregated once more on their
tentative Galerkin matrix): checked against the same composition written
here with scipy and the oracle's standalone aggregation, and by the much
larger a_0 the paper reports for it (Tables 1-2).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.diagnostics import a_numbers
from oracle.oracle import Oracle, aggregate_csr
from paper_2001_11533_gb300 import workloads as W


@pytest.mark.parametrize("N", [9, 17])
def test_geometric_interpolation_reproduces_linear_functions(N):
    w = W.unit_square(N)
    o = Oracle(w, geometric=1, coarse_max=1)
    P = o.scipy("P", 0)
    Nc = (N + 1) // 2
    h, hc = 1.0 / (N - 1), 1.0 / (Nc - 1)
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    ic, jc = np.meshgrid(np.arange(Nc), np.arange(Nc), indexing="xy")
    f = lambda x, y: 0.3 + 1.7 * x - 2.2 * y
    fine = f(i.ravel() * h, j.ravel() * h)
    coarse = f(ic.ravel() * hc, jc.ravel() * hc)
    assert np.abs(P @ coarse - fine).max() <= 1e-14
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)


@pytest.mark.parametrize("N", [9, 17])
def test_geometric_galerkin_equals_coarse_assembly(N):
    Nc = (N + 1) // 2
    fine = Oracle(W.unit_square(N), geometric=1, coarse_max=1)
    direct = Oracle(W.unit_square(Nc), max_levels=1)
    for which in ("A", "My", "Myu", "KN", "Mu"):
        g = fine.scipy(which, 1).toarray()
        d = direct.scipy(which, 0).toarray()
        assert g.shape == d.shape, which
        assert np.abs(g - d).max() <= 1e-13 * np.abs(d).max(), which


def test_geometric_aj_rate_is_a_quarter():
    """a_j / a_j+1 falls towards 1/4 as the level gets finer (Table 1: 0.25-0.29)."""
    o = Oracle(W.unit_square(33), geometric=1, coarse_max=1)
    a = [a_numbers(o, j) for j in range(4)]
    ratios = [a[j][0] / a[j + 1][0] for j in range(3)]
    assert ratios[0] < ratios[1] < ratios[2]
    assert 0.24 <= ratios[0] <= 0.29, ratios
    for av, at in a:   # a~_j approximates a_j (Table 1)
        assert 0.9 <= at / av <= 1.1


def _tentative(agg, nagg):
    n = agg.shape[0]
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nagg))


def test_aggressive_aggregates_are_aggregates_of_aggregates():
    w = W.unit_square(33)   # unjittered: every product below is exact in both orders
    o = Oracle(w, aggressive=1, coarse_max=8)
    A = o.scipy("A", 0)
    agg1, _, n1 = aggregate_csr(A.indptr, A.indices, A.data, 0.08)
    Sh = _tentative(agg1, n1)
    T = (Sh.T @ A @ Sh).tocsr()
    T.sort_indices()
    agg2, _, n2 = aggregate_csr(T.indptr, T.indices, T.data, 0.04)
    got, ng = o.aggregates(0, 0)
    assert ng == n2 and np.array_equal(got, agg2[agg1])
    KN = o.scipy("KN", 0)
    c1, _, m1 = aggregate_csr(KN.indptr, KN.indices, KN.data, 0.08)
    Sc = _tentative(c1, m1)
    TN = (Sc.T @ KN @ Sc).tocsr()
    TN.sort_indices()
    c2, _, m2 = aggregate_csr(TN.indptr, TN.indices, TN.data, 0.04)
    got, ng = o.aggregates(1, 0)
    assert ng == m2 and np.array_equal(got, c2[c1])


def test_aggressive_first_level_has_large_a0():
    """Tables 1-2: aggressive first-level coarsening gives a much larger a_0 and a
    ratio a_0 / a_1 well above one; without it the ratios stay near or below one."""
    w = W.unit_square(33)
    std = Oracle(w, coarse_max=8)
    agg = Oracle(w, aggressive=1, coarse_max=8)
    assert agg.sizes()["state"][1] * 4 < std.sizes()["state"][1]
    a_std = [a_numbers(std, j)[0] for j in range(2)]
    a_agg = [a_numbers(agg, j)[0] for j in range(2)]
    assert a_agg[0] > 2.0 * a_std[0]
    assert a_agg[0] / a_agg[1] > 2.0
    assert a_std[0] / a_std[1] < 1.2


def test_geometric_two_grid_counts_fall_with_n():
    """Shape of Table 5: two-grid outer CG counts fall as h -> 0 for the geometric
    hierarchy and stay at or above them for AMG (beta = 1e-4)."""
    counts = {0: [], 1: []}
    for N in (9, 17, 33):
        w = W.unit_square(N, beta=1e-4, y_d="exact")
        for geo in (0, 1):
            o = Oracle(w, geometric=geo, coarse_max=1, hessian_levels=2, inner_tol=1e-12, mass_tol=1e-12)
            _, _, info = o.solve(precond=1, tol=1e-8)
            counts[geo].append(info["outer_iters"])
    assert counts[1][0] > counts[1][-1] and all(a >= b for a, b in zip(counts[1], counts[1][1:]))
    assert all(g <= a for g, a in zip(counts[1], counts[0]))
