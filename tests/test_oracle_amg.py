"""Pins for the oracle's aggregation hierarchy (Sec. 3.1, smoothed aggregation).

Checked against things other than the oracle's own code: the published
splitmix64 outputs, a brute-force greedy distance-2 independent set and a
parallel-round (Luby-style, fixed priority) construction written here in
Python, the structural properties every aggregation must have, dense numpy
Galerkin triple products (Eq. coarsestiffness, coarsemass), and constant
reproduction of the control prolongator built on the Neumann stiffness.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.oracle import Oracle, aggregate_csr, priority
from paper_2001_11533_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEED = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def test_splitmix64_published_vector():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    s, got = 1234567, []
    for _ in range(5):
        s = (s + SEED) & MASK
        got.append(priority(s ^ SEED))   # priority(i) = mix(SEED ^ i)
    assert got == want


def _strong_graph(A, theta):
    A = A.tocsr()
    d = A.diagonal()
    rows, cols, vals = [], [], []
    for i in range(A.shape[0]):
        for k in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[k]
            a = A.data[k]
            if j != i and a * a >= (theta * theta) * (d[i] * d[j]):
                rows.append(i)
                cols.append(j)
                vals.append(a)
    return sp.csr_matrix((vals, (rows, cols)), shape=A.shape)


def _ball2(G, v):
    out = {v}
    for w in G.indices[G.indptr[v]:G.indptr[v + 1]]:
        out.add(int(w))
        out.update(int(x) for x in G.indices[G.indptr[w]:G.indptr[w + 1]])
    return out


def _greedy_mis2(G):
    n = G.shape[0]
    order = sorted(range(n), key=lambda i: -priority(i))
    covered = np.zeros(n, bool)
    roots = np.zeros(n, bool)
    for v in order:
        if covered[v]:
            continue
        roots[v] = True
        for w in _ball2(G, v):
            covered[w] = True
    return roots


def _parallel_mis2(G):
    """Rounds: an undecided vertex whose priority is the largest among undecided
    vertices within distance 2 becomes a root; then everything within distance 2
    of a new root is removed.  With fixed priorities this is the greedy set."""
    n = G.shape[0]
    pr = [priority(i) for i in range(n)]
    state = np.zeros(n, int)  # 0 undecided, 1 root, 2 removed
    balls = [_ball2(G, v) for v in range(n)]
    while (state == 0).any():
        new = [v for v in range(n) if state[v] == 0 and
               all(pr[v] >= pr[w] for w in balls[v] if state[w] == 0)]
        assert new
        for v in new:
            state[v] = 1
        for v in new:
            for w in balls[v]:
                if state[w] == 0:
                    state[w] = 2
    return state == 1


def _laplacian_5pt(N):
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


def _check_aggregation(A, theta, agg, roots, nagg):
    A = A.tocsr()
    n = A.shape[0]
    G = _strong_graph(A, theta)
    # roots: distance >= 3 pairwise, maximal
    want_roots = _greedy_mis2(G)
    assert np.array_equal(roots, want_roots)
    # every vertex in exactly one aggregate, ids 0..nagg-1 all used
    assert agg.min() >= 0 and agg.max() == nagg - 1
    assert len(np.unique(agg)) == nagg
    # phase 1: root rank ids, strong neighbours of roots share the root's id
    rid = np.cumsum(roots) - 1
    for r in np.flatnonzero(roots):
        assert agg[r] == rid[r]
        for j in G.indices[G.indptr[r]:G.indptr[r + 1]]:
            assert agg[j] == agg[r]
    phase1 = np.full(n, -1)
    for r in np.flatnonzero(roots):
        phase1[r] = rid[r]
        phase1[G.indices[G.indptr[r]:G.indptr[r + 1]]] = rid[r]
    # phase 2: largest |a_ij| among phase-1-aggregated strong neighbours, ties -> smaller id
    nxt = int(roots.sum())
    for i in range(n):
        if phase1[i] >= 0:
            continue
        cand = [(abs(G.data[k]), -phase1[G.indices[k]]) for k in range(G.indptr[i], G.indptr[i + 1])
                if phase1[G.indices[k]] >= 0]
        if cand:
            best = max(cand)
            assert agg[i] == -best[1]
        else:
            assert agg[i] == nxt
            nxt += 1


def test_mis2_parallel_rounds_equal_greedy():
    rng = np.random.default_rng(3)
    for n in (30, 60):
        R = sp.random(n, n, density=0.08, random_state=rng, format="csr")
        G = ((R + R.T) != 0).astype(float)
        G.setdiag(0)
        G.eliminate_zeros()
        G = G.tocsr()
        assert np.array_equal(_parallel_mis2(G), _greedy_mis2(G))


@pytest.mark.parametrize("N", [5, 12])
def test_aggregation_on_grid_laplacian(N):
    A = _laplacian_5pt(N)
    agg, roots, nagg = aggregate_csr(A.indptr, A.indices, A.data, 0.08)
    _check_aggregation(A, 0.08, agg, roots, nagg)


def test_golden_5x5_aggregates():
    """Frozen 5x5 five-point-Laplacian aggregation (written by tests/golden/make_golden.py)."""
    A = _laplacian_5pt(5)
    agg, roots, nagg = aggregate_csr(A.indptr, A.indices, A.data, 0.08)
    lines = [l for l in open(os.path.join(GOLDEN, "agg_laplace5x5.txt")) if not l.startswith("#")]
    want = np.array([int(t) for l in lines for t in l.split()])
    assert np.array_equal(agg, want)
    _check_aggregation(A, 0.08, agg, roots, nagg)


def test_fe_hierarchy_aggregates_valid():
    w = W.lshape_checkerboard(N=33)
    o = Oracle(w, max_levels=3, coarse_max=8)
    sz = o.sizes()
    th = 0.08
    for l in range(sz["Ls"] - 1):
        A = o.scipy("A", l)
        agg, nagg = o.aggregates(0, l)
        _, roots, nagg2 = aggregate_csr(A.indptr, A.indices, A.data, th)
        assert nagg == nagg2
        _check_aggregation(A, th, agg, roots, nagg)
        th *= 0.5


def test_galerkin_products_and_constants():
    w = W.unit_square(17, jitter=0.2, cfg=95)
    w.kappa = np.random.default_rng(4).uniform(1.0, 10.0, w.n_elements)
    o = Oracle(w, max_levels=3, coarse_max=8)
    sz = o.sizes()
    for l in range(sz["Ls"] - 1):
        S = o.scipy("S", l).toarray()
        for name in ("A", "My"):
            F = o.scipy(name, l).toarray()
            Cc = o.scipy(name, l + 1).toarray()
            ref = S.T @ F @ S
            assert np.abs(Cc - ref).max() <= 1e-13 * np.abs(ref).max()
            assert np.array_equal(Cc, Cc.T)
    for l in range(sz["Lc"] - 1):
        P = o.scipy("P", l).toarray()
        # smoothing with the Neumann stiffness keeps constants: P 1 = 1
        assert np.abs(P @ np.ones(P.shape[1]) - 1.0).max() <= 1e-13
        for name in ("KN", "Mu"):
            F = o.scipy(name, l).toarray()
            Cc = o.scipy(name, l + 1).toarray()
            ref = P.T @ F @ P
            assert np.abs(Cc - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(o.scipy("KN", l + 1) @ np.ones(P.shape[1])).max() <= \
            1e-12 * np.abs(o.scipy("KN", l + 1).diagonal()).max()
        one = np.ones(P.shape[1])
        assert one @ (o.scipy("Mu", l + 1) @ one) == pytest.approx(1.0, rel=1e-13)
    for l in range(min(sz["Ls"], sz["Lc"]) - 1):
        S = o.scipy("S", l).toarray()
        P = o.scipy("P", l).toarray()
        ref = S.T @ o.scipy("Myu", l).toarray() @ P
        got = o.scipy("Myu", l + 1).toarray()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_prolongator_definition():
    """S = (I - omega D^-1 A) S_hat with omega = 4/(3 rho), rho = max_i sum_j |a_ij| / a_ii."""
    w = W.unit_square(9, jitter=0.2, cfg=96)
    o = Oracle(w, max_levels=2, coarse_max=4)
    A = o.scipy("A", 0).toarray()
    agg, nagg = o.aggregates(0, 0)
    Sh = np.zeros((A.shape[0], nagg))
    Sh[np.arange(A.shape[0]), agg] = 1.0
    d = np.diag(A)
    rho = (np.abs(A).sum(axis=1) / d).max()
    S = Sh - (4.0 / (3.0 * rho)) * (A / d[:, None]) @ Sh
    assert np.abs(o.scipy("S", 0).toarray() - S).max() <= 1e-14


def test_vcycle_is_spd_and_contracts():
    w = W.unit_square(17, jitter=0.2, cfg=97)
    o = Oracle(w, max_levels=3, coarse_max=8)
    A = o.scipy("A", 0).toarray()
    n = A.shape[0]
    B = np.column_stack([o.vcycle(0, e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    ev = np.linalg.eigvals(B @ A).real
    assert ev.min() > 0.0 and ev.max() < 1.0 + 1e-12   # I - BA has spectrum in [0, 1)
