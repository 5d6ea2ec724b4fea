"""Block solver (the batching pattern in SpMM form): K columns of one problem
advance together, every sparse operator applied to all K in one pass, each
column with its own CG scalars and stopping tests.

Per column the method is the single-column one, so each column must match the
FP64 oracle's single solve (mixed path within 1e-8, FP64 path within 1e-10)
and the block H and Q_0 applies must match the oracle column by column.  The
arithmetic of a column does not depend on the other columns or on the block
width (same grids, same per-column reduction order), so results are compared
bit for bit across widths and with failing neighbours.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(inner_tol=1e-13, mass_tol=1e-13)


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _lshape():
    return W.lshape_checkerboard(N=65)


def _desired_states(w, k):
    """The workload's y_d and smooth variations of it (k columns)."""
    x, y = w.coords[:, 0], w.coords[:, 1]
    base = w.y_d if w.y_d.ndim == 1 else w.y_d[0]
    cols = [base]
    for j in range(1, k):
        cols.append(base * (1.0 + 0.25 * j) + 0.3 * np.sin(np.pi * j * x) * np.cos(np.pi * (j + 1) * y))
    return np.stack(cols)


def _problem(w, **amg):
    from paper_2001_11533_gb300 import amgh
    return amgh.Problem.from_workload(w).amg_setup(**amg)


@pytest.mark.parametrize("precision", [0, 2])
def test_block_hessian_apply_matches_oracle(precision):
    w = _lshape()
    prob = _problem(w, coarse_max=32, precision=precision)
    prob.set_solve_opts(**TIGHT)
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    U = np.random.default_rng(31).standard_normal((3, prob.sizes["n"]))   # K = 4, one padding column
    HU = host(prob.hessian_apply(cuda(U)))
    for u, hu in zip(U, HU):
        assert rel(hu, orc.hessian(u)) <= 1e-10


@pytest.mark.parametrize("precision", [0, 2])
def test_block_precond_apply_matches_oracle(precision):
    w = _lshape()
    prob = _problem(w, coarse_max=32, precision=precision)
    prob.set_solve_opts(**TIGHT)
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    R = np.random.default_rng(32).standard_normal((2, prob.sizes["n"]))
    Z = host(prob.precond_apply(cuda(R)))
    for r, z in zip(R, Z):
        assert rel(z, orc.precond(r)) <= 1e-9


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (2, 1e-8)])
def test_block_solve_matches_oracle(precision, bound):
    w = _lshape()
    Y = _desired_states(w, 5)                        # K = 8, three padding columns
    prob = _problem(w, coarse_max=32, precision=precision)
    u, info, st = prob.solve_block(cuda(Y), tol=1e-12, **TIGHT)
    assert st == 0 and info["status"] == 0 and info["final_relres"] <= 1e-11
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    iters = 0
    for c in range(Y.shape[0]):
        orc.set_yd(Y[c])
        uo, _, io = orc.solve(precond=1, tol=1e-12)
        assert rel(host(u[c]), uo) <= bound, c
        iters += io["outer_iters"]
    assert abs(info["outer_iters"] - iters) <= Y.shape[0]


def test_block_solve_equals_single_solves():
    """Same method per column as amgh_solve: controls agree to the tolerances."""
    w = _lshape()
    Y = _desired_states(w, 3)
    prob = _problem(w, coarse_max=32, precision=2)
    u, info, st = prob.solve_block(cuda(Y), tol=1e-11, inner_tol=1e-12, mass_tol=1e-12)
    assert st == 0
    for c in range(Y.shape[0]):
        prob.set_yd(cuda(Y[c]))
        us, _, _ = prob.solve(tol=1e-11, inner_tol=1e-12, mass_tol=1e-12)
        assert rel(host(u[c]), host(us)) <= 1e-8, c


def test_columns_independent_of_block_width():
    """Each column alone (K = 2 with a padding column) equals the same column
    inside blocks of 4 and 8, bit for bit."""
    w = _lshape()
    Y = _desired_states(w, 6)
    prob = _problem(w, coarse_max=32, precision=2)
    u8, _, st = prob.solve_block(cuda(Y), tol=1e-10)          # K = 8
    assert st == 0
    u4, _, st = prob.solve_block(cuda(Y[:3]), tol=1e-10)      # K = 4
    assert st == 0
    for c in (0, 2, 5):
        u1, _, st = prob.solve_block(cuda(Y[c:c + 1]), tol=1e-10)
        assert st == 0
        assert np.array_equal(host(u1[0]), host(u8[c])), c
        if c < 3:
            assert np.array_equal(host(u4[c]), host(u8[c])), c


def test_failing_and_zero_columns_do_not_disturb_others():
    w = _lshape()
    Y = _desired_states(w, 2)
    prob = _problem(w, coarse_max=32, precision=2)
    clean, _, st = prob.solve_block(cuda(Y), tol=1e-10)
    assert st == 0
    bad = np.array(Y[0])
    interior = np.flatnonzero(w.dirichlet == 0)
    bad[interior[len(interior) // 2]] = np.nan
    mixed = np.stack([Y[0], np.zeros_like(Y[0]), bad, Y[1]])
    u, info, st = prob.solve_block(cuda(mixed), tol=1e-10, raise_on_error=False)
    assert st == -7 and info["status"] == -7                    # NUMERIC: the NaN column
    assert np.array_equal(host(u[0]), host(clean[0]))
    assert np.array_equal(host(u[3]), host(clean[1]))
    assert not np.any(host(u[1]))                               # zero desired state: u = 0


def test_block_level_fallback_matches_oracle():
    # beta = 1.1e-4 on a 65^2 square with 4 Hessian levels: indefinite W-cycle
    w = W.batch_squares(sizes=(65,), per_size=3, rhs=3)[2]
    prob = _problem(w, coarse_max=32)
    _, bad, st = prob.solve_block(cuda(w.y_d), tol=1e-12, raise_on_error=False, **TIGHT)
    assert st == -6
    prob = _problem(w, coarse_max=32)
    u, info, st = prob.solve_block(cuda(w.y_d), tol=1e-12, level_fallback=1, **TIGHT)
    assert st == 0 and info["fallbacks"] >= 1
    orc = Oracle(w, coarse_max=32, hessian_levels=info["hessian_levels"], inner_tol=1e-13, mass_tol=1e-13)
    for c in range(w.y_d.shape[0]):
        orc.set_yd(w.y_d[c])
        uo, _, _ = orc.solve(precond=1, tol=1e-12)
        assert rel(host(u[c]), uo) <= 1e-10, c


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (2, 1e-8)])
def test_block_coarse_cg_matches_oracle(precision, bound):
    """The coarsest level by CG: its right sides shrink with the outer residual,
    so the FP32 V-cycles of precision 2 rely on the per-column power-of-two
    scaling of their input."""
    w = _lshape()
    Y = _desired_states(w, 2)
    prob = _problem(w, coarse_max=32, coarse_solve=1, precision=precision)
    u, info, st = prob.solve_block(cuda(Y), tol=1e-12, coarse_tol=1e-4, **TIGHT)
    assert st == 0 and info["coarse_iters"] > 0
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    orc.set_coarse_solve(1, tol=1e-4)
    for c in range(2):
        orc.set_yd(Y[c])
        uo, _, _ = orc.solve(precond=1, tol=1e-12)
        assert rel(host(u[c]), uo) <= bound, c


def test_batch_block_mode():
    """Batch in block mode equals amgh_solve_block per problem, bit for bit, and
    the per-column batch to the solve tolerance."""
    from paper_2001_11533_gb300 import amgh
    ws = W.batch_squares(sizes=(33, 65), per_size=1, rhs=5)
    opts = dict(coarse_max=600, precision=2)
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs, block=True).setup(**opts)
    us, infos, st = batch.solve([cuda(w.y_d) for w in ws], tol=1e-10)
    batch.close()
    assert st == 0 and all(i["status"] == 0 for i in infos)
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(**opts)
    ucol, _, st = batch.solve([cuda(w.y_d) for w in ws], tol=1e-10)
    batch.close()
    assert st == 0
    for w, u, uc in zip(ws, us, ucol):
        alone = _problem(w, **opts)
        ub, _, st = alone.solve_block(cuda(w.y_d), tol=1e-10)
        assert st == 0 and np.array_equal(host(u), host(ub))
        for c in range(w.y_d.shape[0]):
            assert rel(host(u[c]), host(uc[c])) <= 1e-8


def test_more_columns_than_one_block():
    """10 columns run as a block of 8 and a padded block of 2 more: every
    column still matches the oracle (H applies) and its own one-column block
    solve bit for bit."""
    w = _lshape()
    prob = _problem(w, coarse_max=32, precision=2)
    prob.set_solve_opts(**TIGHT)
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    U = np.random.default_rng(33).standard_normal((10, prob.sizes["n"]))
    HU = host(prob.hessian_apply(cuda(U)))
    for c in (0, 7, 8, 9):
        assert rel(HU[c], orc.hessian(U[c])) <= 1e-10, c
    Y = _desired_states(w, 10)
    u, info, st = prob.solve_block(cuda(Y), tol=1e-10)
    assert st == 0 and info["outer_iters"] > 0
    for c in (1, 8, 9):
        u1, _, st = prob.solve_block(cuda(Y[c:c + 1]), tol=1e-10)
        assert st == 0 and np.array_equal(host(u1[0]), host(u[c])), c


@pytest.mark.parametrize("k", [3, 8])
def test_persistent_mass_cg_matches_graph_replay_and_oracle(k):
    """persistent_cg = 1: the block mass CGs as one cooperative launch each.
    Same arithmetic per row, sums grouped by that launch's blocks: the
    controls agree with the graph-replayed block solve to the CG tolerance
    and with the oracle's single solves per column (mixed bound 1e-8);
    reruns give the same bits."""
    w = _lshape()
    Y = _desired_states(w, k)
    opts = dict(coarse_max=32, precision=2)
    ref = _problem(w, **opts)
    per = _problem(w, persistent_cg=1, **opts)
    sopts = dict(tol=1e-10, inner_tol=1e-12, mass_tol=1e-12)
    u0, i0, st0 = ref.solve_block(cuda(Y), **sopts)
    u1, i1, st1 = per.solve_block(cuda(Y), **sopts)
    assert st0 == 0 and st1 == 0
    assert i1["mass_iters"] > 0
    for c in range(k):
        assert rel(host(u1[c]), host(u0[c])) <= 1e-9, c
    u2, _, st2 = per.solve_block(cuda(Y), **sopts)
    assert st2 == 0 and np.array_equal(host(u1), host(u2))
    orc = Oracle(w, coarse_max=32, **TIGHT)
    for c in (0, k - 1):
        orc.set_yd(Y[c])
        uo, _, _ = orc.solve(precond=1, tol=1e-12)
        assert rel(host(u1[c]), uo) <= 1e-8, c


def test_grid_barriers_time_out_and_recover():
    """Both software grid barriers (the persistent block mass CG and the
    grid-fused V-cycle) driven to give up at their first wait: the call
    returns AMGH_ERR_TIMEOUT, no GPU wait is left hanging, and the next call
    with the default limit gives the clean result bit for bit."""
    from paper_2001_11533_gb300 import amgh
    w = _lshape()
    Y = _desired_states(w, 2)
    per = _problem(w, coarse_max=32, precision=2, persistent_cg=1)
    sopts = dict(tol=1e-10, inner_tol=1e-12, mass_tol=1e-12)
    clean, _, st = per.solve_block(cuda(Y), **sopts)
    assert st == 0
    fused = amgh.Problem.from_workload(w).amg_setup(coarse_max=32, precision=2, fuse_coarse=2)
    fused.set_yd(cuda(Y[0]))
    fclean, _, finfo = fused.solve(tol=1e-10, want_y=False)
    try:
        amgh.debug_grid_polls(0)
        _, _, st = per.solve_block(cuda(Y), raise_on_error=False, **sopts)
        assert st == amgh.ERR_TIMEOUT
        with pytest.raises(amgh.AmghError) as e:
            fused.solve(tol=1e-10, want_y=False)
        assert e.value.code == amgh.ERR_TIMEOUT
    finally:
        amgh.debug_grid_polls(-1)
    again, _, st = per.solve_block(cuda(Y), **sopts)
    assert st == 0 and np.array_equal(host(again), host(clean))
    fagain, _, _ = fused.solve(tol=1e-10, want_y=False)
    assert np.array_equal(host(fagain), host(fclean))
