"""Pin of the oracle's polynomial smoother (the AMG smoother of Sec. 5.2).

Reading of the paper (it names no smoother for its AMG): Chebyshev iteration
of degree k for D^-1 A on [1/30, 1], D the l1 row sums d_i = sum_j |a_ij|,
or k sweeps of l1-Jacobi.  Started from x0 with b = 0, k smoothing steps
multiply the error by E = p_k(D^-1 A), where for Chebyshev

    p_k(t) = T_k((theta - t) / delta) / T_k(theta / delta),
    theta = (1 + 1/30) / 2,  delta = (1 - 1/30) / 2,

the scaled Chebyshev residual polynomial (Saad, Iterative Methods for Sparse
Linear Systems, Sec. 12.3), and p_k(t) = (1 - t)^k for l1-Jacobi.  The test
evaluates T_k in closed form (cos / cosh of k arccos / arccosh) on the
eigenvalues of the symmetric D^-1/2 A D^-1/2, with D computed here from the
assembled matrix, and compares the oracle's smoother, applied to every unit
vector, with that matrix function.  A wrong recurrence coefficient (rho_s and
rho_{s-1} exchanged, theta and delta exchanged, a dropped first step) changes
the polynomial and fails; so does a wrong l1 diagonal.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

LO, HI = 1.0 / 30.0, 1.0


def _cheb_T(k, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(k * np.arccos(x[inside]))
    big = x > 1.0
    out[big] = np.cosh(k * np.arccosh(x[big]))
    neg = x < -1.0
    out[neg] = (-1.0) ** k * np.cosh(k * np.arccosh(-x[neg]))
    return out


def _residual_poly(kind, k, t):
    if kind == "jacobi":
        return (1.0 - t) ** k
    theta, delta = (HI + LO) / 2.0, (HI - LO) / 2.0
    return _cheb_T(k, (theta - t) / delta) / _cheb_T(k, np.array([theta / delta]))[0]


def _propagator(A, kind, k):
    """p_k(D^-1 A) formed through the symmetric similarity D^-1/2 A D^-1/2."""
    d = np.abs(A).sum(axis=1)
    s = 1.0 / np.sqrt(d)
    lam, V = np.linalg.eigh(s[:, None] * A * s[None, :])
    assert lam.min() > 0.0 and lam.max() <= 1.0 + 1e-12   # l1 scaling: spectrum in (0, 1]
    Pm = (V * _residual_poly(kind, k, lam)) @ V.T
    return s[:, None] * Pm / s[None, :]


CASES = [("chebyshev", 2), ("chebyshev", 3), ("chebyshev", 4), ("jacobi", 1), ("jacobi", 2)]


@pytest.mark.parametrize("kind,k", CASES)
def test_error_propagator_is_the_residual_polynomial(kind, k):
    w = W.unit_square(11, jitter=0.2, cfg=131)
    o = Oracle(w, max_levels=2, coarse_max=8, smoother=1 if kind == "chebyshev" else 0, degree=k)
    A = o.scipy("A", 0).toarray()
    n = A.shape[0]
    zero = np.zeros(n)
    E = np.column_stack([o.smooth(0, zero, x0=e) for e in np.eye(n)])
    ref = _propagator(A, kind, k)
    assert np.abs(E - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("kind,k", [("chebyshev", 2), ("jacobi", 2)])
def test_from_zero_is_the_smoothing_operator(kind, k):
    """From x0 = 0: x = (I - p_k(D^-1 A)) A^-1 b, the smoother as an approximate inverse."""
    w = W.unit_square(13, jitter=0.2, cfg=132)
    o = Oracle(w, max_levels=2, coarse_max=8, smoother=1 if kind == "chebyshev" else 0, degree=k)
    A = o.scipy("A", 0).toarray()
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    x = o.smooth(0, b)
    ref = (np.eye(A.shape[0]) - _propagator(A, kind, k)) @ np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def test_chebyshev_minimax_bound():
    """On [1/30, 1] the Chebyshev residual polynomial is bounded by 1/T_k(theta/delta),
    the smallest maximum any degree-k polynomial with p(0) = 1 can reach there."""
    theta, delta = (HI + LO) / 2.0, (HI - LO) / 2.0
    t = np.linspace(LO, HI, 2001)
    for k in (2, 3, 4):
        bound = 1.0 / _cheb_T(k, np.array([theta / delta]))[0]
        assert np.abs(_residual_poly("chebyshev", k, t)).max() <= bound * (1 + 1e-12)
        w = W.unit_square(9, jitter=0.2, cfg=133)
        o = Oracle(w, max_levels=2, coarse_max=8, smoother=1, degree=k)
        A = o.scipy("A", 0).toarray()
        d = np.abs(A).sum(axis=1)
        lam, V = np.linalg.eigh(A / np.sqrt(np.outer(d, d)))
        # eigenvectors of D^-1 A are D^-1/2 V: the smoother scales each by p_k(lambda)
        for j in np.nonzero(lam >= LO)[0]:
            v = V[:, j] / np.sqrt(d)
            got = o.smooth(0, np.zeros_like(v), x0=v)
            gain = np.linalg.norm(got) / np.linalg.norm(v)
            assert gain <= bound * (1 + 1e-9)
