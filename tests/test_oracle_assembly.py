"""Pins for the oracle's P1 assembly (Sec. 2: stiffness and mass matrices).

The oracle assembles with cofactor gradients; these tests check it against
facts that do not come from that code: an independent numpy assembly through
the inverse Jacobian of the affine element map, exact integrals of linear
functions (the P1 mass matrix integrates products of P1 functions exactly),
the constant null space of the Neumann stiffness, and harmonicity of linear
functions for kappa = 1.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W


def _independent_assembly(w):
    """Dense K, M from reference-element gradients and inv(J) (not the oracle's formula)."""
    d = w.dim
    n = w.n_vertices
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    ref_grad = np.vstack([-np.ones((1, d)), np.eye(d)])      # (d+1, d) gradients on the reference simplex
    import math
    ref_mass = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    for e, ev in enumerate(w.elements):
        P = w.coords[ev]
        J = (P[1:] - P[0]).T                                 # columns e_k
        vol = abs(np.linalg.det(J)) / math.factorial(d)
        G = ref_grad @ np.linalg.inv(J)                      # rows grad(lambda_k)
        K[np.ix_(ev, ev)] += w.kappa[e] * vol * (G @ G.T)
        M[np.ix_(ev, ev)] += vol * ref_mass
    return K, M


def _small_cases():
    sq = W.unit_square(6, jitter=0.2, cfg=91)
    sq.kappa = np.random.default_rng(5).uniform(0.5, 3.0, sq.n_elements)
    c, e = W.grid3d_kuhn(4)
    cube = W.Workload("cube4", 3, c, e, W.boundary_vertices(e, c.shape[0]),
                      np.random.default_rng(6).uniform(0.5, 3.0, e.shape[0]), 1e-2,
                      np.zeros(c.shape[0]))
    return [sq, cube]


@pytest.mark.parametrize("case", [0, 1])
def test_matches_independent_assembly(case):
    w = _small_cases()[case]
    o = Oracle(w, setup=False)
    Kd, Md = _independent_assembly(w)
    K = o.scipy("Kfull").toarray()
    M = o.scipy("Mfull").toarray()
    assert np.abs(K - Kd).max() <= 1e-12 * np.abs(Kd).max()
    assert np.abs(M - Md).max() <= 1e-12 * np.abs(Md).max()


def test_sorted_symmetric_pattern_and_values():
    w = W.lshape_checkerboard(N=33)
    o = Oracle(w, setup=False)
    for name in ("Kfull", "Mfull"):
        rp, ci, v, shape = o.matrix(name)
        for i in range(shape[0]):
            row = ci[rp[i]:rp[i + 1]]
            assert (np.diff(row) > 0).all()
        A = o.scipy(name)
        # exactly symmetric: same element contributions in the same order
        assert (A != A.T).nnz == 0


@pytest.mark.parametrize("maker", ["lshape", "square", "cube"])
def test_exact_integrals(maker):
    if maker == "lshape":
        w = W.lshape_checkerboard(N=33)
        area, ix2, ixy = 0.75, 3.0 / 16.0, 1.0 / 4.0 - 0.25 * 0.75 * 0.75
    elif maker == "square":
        w = W.unit_square(17, jitter=0.2, cfg=92)
        area, ix2, ixy = 1.0, 1.0 / 3.0, 0.25
    else:
        c, e = W.grid3d_kuhn(5)
        w = W.Workload("cube5", 3, c, e, W.boundary_vertices(e, c.shape[0]),
                       np.ones(e.shape[0]), 1e-2, np.zeros(c.shape[0]))
        area, ix2, ixy = 1.0, 1.0 / 3.0, 0.25
    o = Oracle(w, setup=False)
    M = o.scipy("Mfull")
    one = np.ones(w.n_vertices)
    x = w.coords[:, 0]
    y = w.coords[:, 1]
    assert one @ (M @ one) == pytest.approx(area, rel=1e-13)
    assert x @ (M @ x) == pytest.approx(ix2, rel=1e-13)
    assert x @ (M @ y) == pytest.approx(ixy, rel=1e-13)
    # stiffness: energy of the linear function x is sum_T kappa_T |T|
    K = o.scipy("Kfull")
    vol = W.element_measure(w.coords, w.elements)
    assert x @ (K @ x) == pytest.approx(float((w.kappa * vol).sum()), rel=1e-12)
    # constant null space of the all-vertex (Neumann) stiffness
    assert np.abs(K @ one).max() <= 1e-12 * abs(K.diagonal()).max()


def test_linear_functions_harmonic():
    """kappa = 1: the P1 stiffness maps a linear function to zero at interior vertices."""
    w = W.unit_square(9, jitter=0.2, cfg=93)
    o = Oracle(w, setup=False)
    K = o.scipy("Kfull")
    interior = w.dirichlet == 0
    for f in (w.coords[:, 0], w.coords[:, 1], 2 * w.coords[:, 0] - 3 * w.coords[:, 1] + 1):
        r = K @ f
        assert np.abs(r[interior]).max() <= 1e-12


def test_state_restriction():
    """A, M_y are the interior rows/cols and M_yu the interior rows of the full matrices."""
    w = W.unit_square(9, jitter=0.2, cfg=94)
    o = Oracle(w, max_levels=1)
    K = o.scipy("Kfull").toarray()
    M = o.scipy("Mfull").toarray()
    st = np.flatnonzero(w.dirichlet == 0)
    assert np.array_equal(o.scipy("A").toarray(), K[np.ix_(st, st)])
    assert np.array_equal(o.scipy("My").toarray(), M[np.ix_(st, st)])
    assert np.array_equal(o.scipy("Myu").toarray(), M[st, :])
    assert np.array_equal(o.scipy("Mu").toarray(), M)
    assert np.array_equal(o.scipy("KN").toarray(), K)


def test_all_dirichlet_mesh_rejected():
    """A mesh whose every vertex lies on the Dirichlet boundary has no state
    space (y = 0 for every control), so the problem of Sec. 2 is rejected."""
    import pytest
    from oracle.oracle import Oracle, OracleError
    w = W.unit_square(2)
    assert w.n_interior == 0
    with pytest.raises(OracleError):
        Oracle(w)


def test_kuhn_cell_stiffness_is_scaled_tridiagonal():
    """Every Kuhn tetrahedron of the structured cube has the P1 stiffness
    kappa_T h/6 tridiag(-1, [1 2 2 1], -1) in path order (the closed form the
    matrix-free operator applies): one cell, six tetrahedra with different
    kappa, against the oracle's assembly."""
    import itertools
    from oracle.oracle import Oracle
    for N in (2, 3):
        coords, elems = W.grid3d_kuhn(N)
        h = 1.0 / (N - 1)
        kappa = 1.0 + np.arange(elems.shape[0]) * 0.37
        w = W.Workload("kuhn", 3, coords, elems, np.zeros(coords.shape[0], np.uint8), kappa, 1.0,
                       np.zeros(coords.shape[0]), {})
        o = Oracle(w, setup=False)
        K = o.scipy("Kfull").toarray()
        T = np.array([[1, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 1]], float)
        ref = np.zeros_like(K)
        for e, ev in enumerate(elems):
            ref[np.ix_(ev, ev)] += kappa[e] * h / 6.0 * T
        assert np.abs(K - ref).max() <= 1e-14 * np.abs(ref).max()
