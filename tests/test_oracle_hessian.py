"""Pins for the oracle's reduced Hessian, right side, gradient and outer CG.

References that are not the oracle's code: dense numpy/LAPACK solves of the
KKT system and of H = M_yu^T A^-1 M_y A^-1 M_yu + beta M_u (Sec. 2 and
Eq. firstorderpractice), the closed-form continuous optimum (2D analogue of
Sec. 5.3's Eq. test-state), symmetry / coercivity identities of H, central
differences of the quadratic reduced cost, and the mesh-independent iteration
count of unpreconditioned CG (Sec. 1, Table 4).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W


def _dense(o):
    A = o.scipy("A").toarray()
    My = o.scipy("My").toarray()
    Myu = o.scipy("Myu").toarray()
    Mu = o.scipy("Mu").toarray()
    return A, My, Myu, Mu


def _case(N=9, beta=1e-2, cfg=98):
    w = W.unit_square(N, beta=beta, jitter=0.2, cfg=cfg)
    w.kappa = np.random.default_rng(cfg).uniform(1.0, 20.0, w.n_elements)
    w.y_d = np.random.default_rng(cfg + 1).standard_normal(w.n_vertices)
    return w


def test_hessian_matches_dense():
    w = _case(9)
    o = Oracle(w, max_levels=3, coarse_max=8, inner_tol=1e-14)
    A, My, Myu, Mu = _dense(o)
    H = Myu.T @ np.linalg.solve(A, My @ np.linalg.solve(A, Myu)) + w.beta * Mu
    for u in np.random.default_rng(0).standard_normal((5, w.n_vertices)):
        hu = o.hessian(u)
        assert np.linalg.norm(hu - H @ u) <= 1e-11 * np.linalg.norm(H @ u)
    b = o.rhs()
    yd = w.y_d[w.dirichlet == 0]
    bref = Myu.T @ np.linalg.solve(A, My @ yd)
    assert np.linalg.norm(b - bref) <= 1e-11 * np.linalg.norm(bref)


def test_kkt_direct_solve():
    """u from outer CG equals the KKT solution [[My,0,A],[0,bMu,-Myu^T],[A,-Myu,0]]."""
    for N, beta, levels in ((5, 1e-2, 3), (9, 1e-4, 2), (17, 1e-2, 3)):
        w = W.unit_square(N, beta=beta, y_d="sin")
        o = Oracle(w, max_levels=levels, coarse_max=4, inner_tol=1e-14, mass_tol=1e-14)
        A, My, Myu, Mu = _dense(o)
        m, n = A.shape[0], Mu.shape[0]
        Z = np.zeros
        K = np.block([[My, Z((m, n)), A],
                      [Z((n, m)), beta * Mu, -Myu.T],
                      [A, -Myu, Z((m, m))]])
        yd = w.y_d[w.dirichlet == 0]
        rhs = np.concatenate([My @ yd, Z(n), Z(m)])
        sol = np.linalg.solve(K, rhs)
        y_k, u_k = sol[:m], sol[m:m + n]
        u, y, info = o.solve(precond=1, tol=1e-13)
        assert np.linalg.norm(u - u_k) <= 1e-11 * np.linalg.norm(u_k), info
        assert np.linalg.norm(y - y_k) <= 1e-11 * np.linalg.norm(y_k)


def test_indefinite_multilevel_is_reported():
    """Too many levels at small beta can make W indefinite (Sec. 3.2, Sec. 5.6); CG
    must stop with INDEFINITE instead of returning garbage."""
    from oracle.oracle import INDEFINITE, OracleError
    w = W.unit_square(9, beta=1e-4, y_d="sin")
    o = Oracle(w, max_levels=3, coarse_max=4, inner_tol=1e-14, mass_tol=1e-14)
    Q = np.column_stack([o.precond(e) for e in np.eye(o.n)])
    assert np.linalg.eigvalsh(0.5 * (Q + Q.T)).min() < 0.0
    with pytest.raises(OracleError) as ei:
        o.solve(precond=1, tol=1e-13)
    assert ei.value.code == INDEFINITE
    # the two-grid preconditioner (2 levels) is always positive definite (Sec. 3.1)
    o2 = Oracle(w, max_levels=2, coarse_max=4, inner_tol=1e-14, mass_tol=1e-14)
    Q2 = np.column_stack([o2.precond(e) for e in np.eye(o2.n)])
    assert np.linalg.eigvalsh(0.5 * (Q2 + Q2.T)).min() > 0.0


def test_hessian_symmetric_coercive():
    w = _case(17, beta=1e-3, cfg=99)
    o = Oracle(w, max_levels=3, coarse_max=8, inner_tol=1e-14)
    Mu = o.scipy("Mu")
    V = np.random.default_rng(1).standard_normal((6, w.n_vertices))
    H = [o.hessian(v) for v in V]
    hnorm = max(np.linalg.norm(h) / np.linalg.norm(v) for h, v in zip(H, V))
    for i in range(len(V)):
        for j in range(i + 1, len(V)):
            a, b = V[i] @ H[j], V[j] @ H[i]
            assert abs(a - b) <= 1e-12 * hnorm * np.linalg.norm(V[i]) * np.linalg.norm(V[j])
        # (G u, u)_{M_u} >= beta (u, u)_{M_u}   (coercivity used in Lemma 2)
        assert V[i] @ H[i] >= w.beta * (V[i] @ (Mu @ V[i]))


def test_adjoint_consistency():
    """w^T M_y (A^-1 M_yu u) = (M_yu^T A^-T M_y w)^T u  (Sec. 2, adjoint K*)."""
    w = _case(17, cfg=100)
    o = Oracle(w, max_levels=3, coarse_max=8)
    My, Myu = o.scipy("My"), o.scipy("Myu")
    rng = np.random.default_rng(2)
    for _ in range(3):
        u = rng.standard_normal(o.n)
        z = rng.standard_normal(o.m)
        y, _ = o.state_solve(Myu @ u, tol=1e-14)
        p, _ = o.state_solve(My @ z, tol=1e-14)
        lhs = z @ (My @ y)
        rhs = (Myu.T @ p) @ u
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-15


def test_closed_form_second_order():
    """y_d = (1/(2pi^2) + 2 pi^2 beta) sin sin gives u* = sin(pi x) sin(pi y)."""
    beta = 1e-2
    errs = []
    for N in (17, 33, 65, 129):
        w = W.unit_square(N, beta=beta, y_d="exact")
        o = Oracle(w, coarse_max=32)
        u, y, info = o.solve(precond=1, tol=1e-12)
        ustar = np.sin(np.pi * w.coords[:, 0]) * np.sin(np.pi * w.coords[:, 1])
        e = u - ustar
        errs.append(np.sqrt(e @ (o.scipy("Mu") @ e)))
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    assert all(3.6 <= r <= 4.4 for r in ratios), (errs, ratios)


def test_tiny_case_value():
    """33x33, beta=1e-2, y_d = sin sin: u ~ sin sin / (1/(2pi^2) + 2 pi^2 beta) to O(h^2)."""
    w = W.tiny_fp64()
    o = Oracle(w, max_levels=3, coarse_max=16)
    assert o.sizes()["Ls"] == 3
    u, y, info = o.solve(precond=1, tol=1e-10)
    c = 1.0 / (1.0 / (2 * np.pi ** 2) + 2 * np.pi ** 2 * 1e-2)
    ustar = c * np.sin(np.pi * w.coords[:, 0]) * np.sin(np.pi * w.coords[:, 1])
    assert np.abs(u - ustar).max() <= 0.02 * c
    assert info["relres"] <= 1e-10


def test_gradient_central_differences():
    """J is quadratic, so the central difference equals grad J . d up to rounding;
    the step 1e-3 keeps the rounding term eps_mach |J| / step far below 1e-6."""
    w = _case(17, beta=1e-3, cfg=101)
    o = Oracle(w, max_levels=3, coarse_max=8, inner_tol=1e-14)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(o.n)
    J0, _, g = o.objective(u)
    eps = 1e-3
    for _ in range(5):
        d = rng.standard_normal(o.n)
        d /= np.linalg.norm(d)
        Jp, _, _ = o.objective(u + eps * d, grad=False)
        Jm, _, _ = o.objective(u - eps * d, grad=False)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(g @ d) + 1e-14 * abs(J0) / eps
    # gradient = H u - b
    hb = o.hessian(u) - o.rhs()
    assert np.linalg.norm(g - hb) <= 1e-10 * np.linalg.norm(g)


def test_gradient_vanishes_at_optimum():
    w = W.unit_square(17, beta=1e-2, y_d="sin")
    o = Oracle(w, coarse_max=8, inner_tol=1e-13)
    u, y, info = o.solve(precond=1, tol=1e-12)
    _, _, g = o.objective(u)
    assert np.linalg.norm(g) <= 1e-10 * np.linalg.norm(o.rhs())


def test_unpreconditioned_mesh_independent():
    """Unpreconditioned outer CG needs a number of iterations bounded independently
    of h (Sec. 1).  On the 2D square with a smooth y_d the count falls and then
    settles, so the pin is: no growth past the coarsest mesh, and the two finest
    meshes within 20% of each other."""
    its = []
    for N in (17, 33, 65, 129, 257):
        w = W.unit_square(N, beta=1e-2, y_d="sin")
        o = Oracle(w, coarse_max=32)
        _, _, info = o.solve(precond=0, tol=1e-8)
        its.append(info["outer_iters"])
    assert max(its) <= its[0], its
    assert max(its[-2:]) <= 1.2 * min(its[-2:]), its


def test_preconditioned_fewer_and_not_growing():
    """Multilevel / two-grid PCG needs far fewer iterations than plain CG and the
    count does not grow with N (Tables 3 and 5).  At beta = 1e-4 on the square the
    W-cycle with 3+ levels is indefinite (the caveat of Sec. 3.2), so that beta is
    pinned with the two-grid preconditioner, which is always definite."""
    for beta, levels, sizes in ((1e-2, 25, (33, 65, 129, 257)), (1e-4, 2, (17, 33, 65))):
        pre, non = [], []
        for N in sizes:
            w = W.unit_square(N, beta=beta, y_d="sin")
            o = Oracle(w, coarse_max=32, max_levels=levels)
            pre.append(o.solve(precond=1, tol=1e-8)[2]["outer_iters"])
            non.append(o.solve(precond=0, tol=1e-8)[2]["outer_iters"])
        assert all(p < q for p, q in zip(pre, non)), (beta, pre, non)
        assert 1.5 * pre[-1] <= non[-1], (beta, pre, non)
        assert max(pre[1:]) <= pre[0], (beta, pre)


def test_openmp_build_is_bit_identical():
    """The -fopenmp build (multi-core CPU timing) splits only row loops, so its
    Hessian apply and preconditioner equal the sequential build's bit for bit,
    on a mesh large enough for the threaded branch to run."""
    from oracle import oracle as orc_mod
    w = W.unit_square(161, beta=1e-3, jitter=0.2, cfg=151)
    u = np.random.default_rng(7).standard_normal(w.n_vertices)
    res = []
    for omp in (False, True):
        o = Oracle(w, coarse_max=200, omp=omp)
        res.append((o.hessian(u), o.precond(u)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert orc_mod.threads(False) == 1
