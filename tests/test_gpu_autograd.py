"""Differentiation pattern: torch.autograd.Function over the C ABI.

The reduced cost J(u) is quadratic, so its central difference equals the
directional derivative up to rounding of J itself; the adjoint gradient is
also compared with the FP64 oracle's, and the state solve's backward with the
adjoint identity <ybar, K u> = <K^T ybar, u> (Sec. 2).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TIGHT = dict(inner_tol=1e-13, mass_tol=1e-13)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _problem(w, **opts):
    from paper_2001_11533_gb300 import amgh
    p = amgh.Problem.from_workload(w).amg_setup(**opts)
    p.set_solve_opts(**TIGHT)
    return p


def test_gradient_matches_oracle_3d():
    import torch
    from paper_2001_11533_gb300.autograd import reduced_cost
    w = W.cube_grf(N=9, features=64)
    prob = _problem(w, coarse_max=16)
    orc = Oracle(w, coarse_max=16, inner_tol=1e-13)
    u0 = np.random.default_rng(31).standard_normal(w.n_vertices)
    u = _cuda(u0).requires_grad_(True)
    J = reduced_cost(u, prob)
    J.backward()
    Jo, _, go = orc.objective(u0)
    assert abs(J.item() - Jo) <= 1e-11 * abs(Jo)
    g = u.grad.cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-10 * np.linalg.norm(go)


def test_state_solve_backward_is_adjoint():
    import torch
    from paper_2001_11533_gb300.autograd import state_solve
    w = W.lshape_checkerboard(N=65)
    prob = _problem(w, coarse_max=32)
    rng = np.random.default_rng(32)
    u = _cuda(rng.standard_normal(w.n_vertices)).requires_grad_(True)
    ybar = _cuda(rng.standard_normal(w.n_interior))
    y = state_solve(u, prob)
    (y * ybar).sum().backward()
    lhs = float((ybar * y.detach()).sum())
    rhs = float((u.grad * u.detach()).sum())
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-30)


@pytest.mark.slow
def test_central_differences_full_cube_129():
    """129^3 Kuhn cube, kappa = exp(GRF), beta = 1e-5: 20 seeded directions, step
    1e-6.  J is quadratic, so |fd - g.d| is bounded by the rounding and solve error
    of J divided by the step."""
    import torch
    from paper_2001_11533_gb300.autograd import reduced_cost
    w = W.cube_grf(N=129, features=64)
    prob = _problem(w, precision=2)
    n = w.n_vertices
    u = _cuda(W.random_vectors(n, 1, 2, 6)[0]).requires_grad_(True)
    J = reduced_cost(u, prob)
    J.backward()
    g = u.grad.detach()
    D = W.random_vectors(n, 20, 2, 5)
    h = 1e-6
    rel_err, j_err = [], []
    for d in D:
        d = _cuda(d / np.linalg.norm(d))
        with torch.no_grad():
            jp = reduced_cost(u.detach() + h * d, prob).item()
            jm = reduced_cost(u.detach() - h * d, prob).item()
        fd = (jp - jm) / (2 * h)
        gd = float((g * d).sum())
        rel_err.append(abs(fd - gd) / abs(gd))
        # J is quadratic: fd - g.d is the error of the two values of J (rounding
        # and the inner solves' tolerance, 1e-13 relative) divided by 2h
        j_err.append(abs(fd - gd) * 2 * h / abs(J.item()))
    # with the step of the workload (1e-6) the difference J(u+hd) - J(u-hd) is
    # ~1e-10 |J| for these unit directions, so rounding of J (~1e-16 |J|) alone
    # limits |fd - g.d| / |g.d| to ~1e-6 .. 1e-2: the check is that fd - g.d is
    # at the rounding level of J.  Because J is exactly quadratic, the same
    # difference with a step of 0.1 is exact up to rounding 1e5 times smaller
    # relative to g.d, and must then match g.d to 1e-6.
    big = []
    for d in D[:5]:
        d = _cuda(d / np.linalg.norm(d))
        with torch.no_grad():
            jp = reduced_cost(u.detach() + 0.1 * d, prob).item()
            jm = reduced_cost(u.detach() - 0.1 * d, prob).item()
        gd = float((g * d).sum())
        big.append(abs((jp - jm) / 0.2 - gd) / abs(gd))
    print(f"central differences, 20 directions, step 1e-6: worst |fd - g.d|/|g.d| = {max(rel_err):.3e}, "
          f"worst |fd - g.d| 2h/|J| = {max(j_err):.3e} (|J| = {J.item():.6e}); "
          f"5 directions, step 0.1: worst |fd - g.d|/|g.d| = {max(big):.3e}")
    assert max(j_err) <= 1e-14, (max(rel_err), max(j_err))
    assert max(big) <= 1e-6, big
