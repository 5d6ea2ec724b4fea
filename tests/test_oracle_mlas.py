"""Pins for the oracle's Hessian preconditioner (Sec. 3.1, 3.2 and 5.2).

Dense references built here with numpy from the oracle's level matrices:
the two-grid T (Eq. twogriddirect) and its claimed inverse (Eq. twogrid), the
projection identities of P Pi (Sec. 3.1), the M_u-scaled form
T^-1 M_u^-1 = P H_H^-1 P^T + beta^-1 (M_u^-1 - P M_{u,H}^-1 P^T) (Sec. 5.2), and
the MLAS recursion against the closed formula W_j = 2 T_j^-1 - T_j^-1 G_j T_j^-1
(Eq. twogridinmultiactual, Algorithm MLAS).
"""
import numpy as np

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W


def _levels(o, ell):
    L = []
    for j in range(ell):
        A = o.scipy("A", j).toarray()
        My = o.scipy("My", j).toarray()
        Myu = o.scipy("Myu", j).toarray()
        Mu = o.scipy("Mu", j).toarray()
        H = Myu.T @ np.linalg.solve(A, My @ np.linalg.solve(A, Myu)) + o.w.beta * Mu
        P = o.scipy("P", j).toarray() if j + 1 < ell else None
        L.append({"Mu": Mu, "H": H, "P": P})
    return L


def _case(N, beta, levels, cfg=120):
    w = W.unit_square(N, beta=beta, jitter=0.2, cfg=cfg)
    w.kappa = np.random.default_rng(cfg).uniform(1.0, 5.0, w.n_elements)
    return Oracle(w, max_levels=levels, coarse_max=8, inner_tol=1e-14, mass_tol=1e-14)


def test_two_grid_inverse_and_projection():
    o = _case(17, 1e-2, 2)
    assert o.sizes()["ell"] == 2
    L = _levels(o, 2)
    beta = o.w.beta
    Mu, H, P = L[0]["Mu"], L[0]["H"], L[0]["P"]
    MuH, HH = L[1]["Mu"], L[1]["H"]
    n = Mu.shape[0]
    Pi = np.linalg.solve(MuH, P.T @ Mu)                      # L2 projection
    PPi = P @ Pi
    assert np.abs(Pi @ P - np.eye(P.shape[1])).max() <= 1e-10
    assert np.abs(PPi @ PPi - PPi).max() <= 1e-10
    G = np.linalg.solve(Mu, H)
    GH = np.linalg.solve(MuH, HH)
    T = P @ GH @ Pi + beta * (np.eye(n) - PPi)
    Tinv = P @ np.linalg.solve(GH, Pi) + (np.eye(n) - PPi) / beta
    assert np.abs(T @ Tinv - np.eye(n)).max() <= 1e-8
    # M_u-scaled form used in practice
    R = P @ np.linalg.solve(HH, P.T) + (np.linalg.inv(Mu) - P @ np.linalg.solve(MuH, P.T)) / beta
    assert np.abs(Tinv @ np.linalg.inv(Mu) - R).max() <= 1e-8 * np.abs(R).max()
    Ro = np.column_stack([o.precond(e) for e in np.eye(n)])
    assert np.abs(Ro - R).max() <= 1e-9 * np.abs(R).max()
    # two-grid is symmetric positive definite
    assert np.linalg.eigvalsh(0.5 * (Ro + Ro.T)).min() > 0
    # and a good preconditioner: spectrum of R H clustered around 1
    ev = np.linalg.eigvals(R @ H).real
    assert ev.min() > 0.3 and ev.max() < 2.0
    _ = G


def test_mlas_matches_closed_formula():
    o = _case(33, 1e-1, 4, cfg=121)
    ell = o.sizes()["ell"]
    assert ell >= 3
    L = _levels(o, ell)
    beta = o.w.beta
    Q = [None] * ell
    Q[ell - 1] = np.linalg.inv(L[ell - 1]["H"])
    Rs = [None] * ell
    for j in range(ell - 2, -1, -1):
        P, Mu, MuH = L[j]["P"], L[j]["Mu"], L[j + 1]["Mu"]
        R = P @ Q[j + 1] @ P.T + (np.linalg.inv(Mu) - P @ np.linalg.solve(MuH, P.T)) / beta
        Rs[j] = R
        Q[j] = R if j == 0 else 2 * R - R @ L[j]["H"] @ R
    rng = np.random.default_rng(8)
    for _ in range(3):
        b = rng.standard_normal(o.n)
        z = o.precond(b)
        assert np.linalg.norm(z - Q[0] @ b) <= 1e-9 * np.linalg.norm(Q[0] @ b)
    for j in range(1, ell - 1):
        bj = rng.standard_normal(L[j]["Mu"].shape[0])
        assert np.linalg.norm(o.precond(bj, level=j) - Q[j] @ bj) <= 1e-9 * np.linalg.norm(Q[j] @ bj)
        assert np.linalg.norm(o.R(bj, level=j) - Rs[j] @ bj) <= 1e-9 * np.linalg.norm(Rs[j] @ bj)


def test_coarsest_cg_solves_the_coarse_hessian():
    """Coarsest level by plain CG (Sec. 5.2): the residual meets the coarse
    tolerance against a dense numpy H_{ell-1}; a tight tolerance gives H^-1 b."""
    o = _case(17, 1e-2, 3)
    o.set_precond_tol(1e-14)
    ell = o.sizes()["ell"]
    assert ell == 3
    H = _levels(o, ell)[ell - 1]["H"]
    b = np.random.default_rng(5).standard_normal(H.shape[0])
    o.set_coarse_solve(1, tol=1e-4)
    x = o.precond(b, level=ell - 1)
    its = o.set_coarse_solve(1, tol=1e-4)
    assert its >= 2
    assert np.linalg.norm(b - H @ x) <= 1.0001e-4 * np.linalg.norm(b)
    o.set_coarse_solve(1, tol=1e-13)
    x = o.precond(b, level=ell - 1)
    xd = np.linalg.solve(H, b)
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    # and the whole W-cycle then equals the one with the dense coarse inverse
    r = np.random.default_rng(6).standard_normal(o.n)
    z_cg = o.precond(r)
    o.set_coarse_solve(0)
    z_dense = o.precond(r)
    assert np.abs(z_cg - z_dense).max() <= 1e-9 * np.abs(z_dense).max()


def test_solution_does_not_depend_on_the_coarse_solve():
    w = W.unit_square(33, beta=1e-3, jitter=0.2, cfg=121)
    o = Oracle(w, coarse_max=16, inner_tol=1e-13, mass_tol=1e-13)
    assert o.sizes()["ell"] >= 3
    u_dense, _, _ = o.solve(tol=1e-11)
    o.set_coarse_solve(1, tol=1e-4)
    u_cg, _, info = o.solve(tol=1e-11)
    assert np.abs(u_cg - u_dense).max() <= 1e-8 * np.abs(u_dense).max()
