"""Dense a_j and a~_j of the multilevel analysis, from the oracle's hierarchy.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain numpy on dense
matrices, for the small meshes of the tests.  With K_j = A_j^-1 M_yu,j the
control-to-state map on level j (Eq. solutionopdef on that level), S_j the
state interpolation, P_j the control interpolation and
Pi_j = M_u,j+1^-1 P_j^T M_u,j the L2 projection onto the coarse control space
(Eq. for the projection in Sec. 3.1), the two-level approximation numbers are
    a_j  = || M_y,j^1/2 (K_j - S_j K_j+1 Pi_j) M_u,j^-1/2 ||_2   (Eq. ajnumerical)
    a~_j = || K_j - S_j K_j+1 Pi_j ||_2                             (Eq. aj-tilde)
and the rate of Eq. ajdecreaserate is estimated by a_j / a_j+1 (Tables 1-2).
"""
from __future__ import annotations

import numpy as np


def _sym_power(M, p):
    """M^p for a symmetric positive definite matrix, by its eigendecomposition."""
    lam, V = np.linalg.eigh(M)
    return (V * lam ** p) @ V.T


def two_level_difference(orc, j):
    """D_j = K_j - S_j K_j+1 Pi_j (dense, m_j x n_j), with M_y,j and M_u,j."""
    A = orc.scipy("A", j).toarray()
    My = orc.scipy("My", j).toarray()
    Myu = orc.scipy("Myu", j).toarray()
    Mu = orc.scipy("Mu", j).toarray()
    S = orc.scipy("S", j).toarray()
    P = orc.scipy("P", j).toarray()
    A1 = orc.scipy("A", j + 1).toarray()
    Myu1 = orc.scipy("Myu", j + 1).toarray()
    Mu1 = orc.scipy("Mu", j + 1).toarray()
    K = np.linalg.solve(A, Myu)
    K1 = np.linalg.solve(A1, Myu1)
    Pi = np.linalg.solve(Mu1, P.T @ Mu)
    return K - S @ K1 @ Pi, My, Mu


def a_numbers(orc, j):
    """(a_j, a~_j) of Eq. ajnumerical and Eq. aj-tilde on level j."""
    D, My, Mu = two_level_difference(orc, j)
    a = np.linalg.norm(_sym_power(My, 0.5) @ D @ _sym_power(Mu, -0.5), 2)
    return float(a), float(np.linalg.norm(D, 2))
