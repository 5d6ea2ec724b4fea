"""The single-column persistent mass CG (persistent_cg = 1, precision 2).

Every mass solve of the mixed form runs its iterations in one cooperative
launch (the block solver's K = 1 kernels, two bounded grid barriers per
iteration).  Same method per element; the sums are grouped by the launch's
blocks, so the results agree with the graph-replayed solve to the CG
tolerance, and with the oracle within the mixed bound; reruns give the same
bits.  The batch runtime, whose handles run beside each other, keeps
cooperative launches off.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_mass_solves_match_graph_replay_and_oracle():
    import torch
    from paper_2001_11533_gb300 import amgh
    w = W.lshape_checkerboard(N=65)
    opts = dict(coarse_max=32, precision=2)
    ref = amgh.Problem.from_workload(w).amg_setup(**opts)
    per = amgh.Problem.from_workload(w).amg_setup(persistent_cg=1, **opts)
    b = torch.from_numpy(np.random.default_rng(7).standard_normal(ref.sizes["n"])).cuda()
    tight = dict(tol=1e-10, inner_tol=1e-12, mass_tol=1e-12)
    for prob in (ref, per):
        prob.set_solve_opts(inner_tol=1e-12, mass_tol=1e-12)
    for lvl in range(min(ref.sizes["Lc"], 3)):
        nl = ref.sizes["control"][lvl]
        x0, it0 = ref.mass_solve(lvl, b[:nl].contiguous())
        x1, it1 = per.mass_solve(lvl, b[:nl].contiguous())
        assert it1 > 0 and abs(it1 - it0) <= 2, (lvl, it0, it1)
        assert rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-10, lvl
    u0, _, i0 = ref.solve(want_y=False, **tight)
    u1, _, i1 = per.solve(want_y=False, **tight)
    assert i1["mass_iters"] > 0 and abs(i1["outer_iters"] - i0["outer_iters"]) <= 1
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-9
    u2, _, _ = per.solve(want_y=False, **tight)
    assert np.array_equal(u1.cpu().numpy(), u2.cpu().numpy())
    orc = Oracle(w, coarse_max=32, inner_tol=1e-13, mass_tol=1e-13)
    uo, _, _ = orc.solve(precond=1, tol=1e-12)
    assert rel(u1.cpu().numpy(), uo) <= 1e-8


def test_batch_keeps_cooperative_launches_off():
    """persistent_cg and fuse_coarse = 2 passed to a batch setup: its solves
    equal those of a batch set up without them, bit for bit."""
    import torch
    from paper_2001_11533_gb300 import amgh
    ws = W.batch_squares(sizes=(65,), per_size=2, rhs=3)
    yds = [torch.from_numpy(np.ascontiguousarray(w.y_d)).cuda() for w in ws]
    sopts = dict(tol=1e-8, inner_tol=1e-10, mass_tol=1e-8, precond_tol=1e-8, level_fallback=1)
    amg = dict(coarse_max=1000, precision=2, coarse_solve=2)
    plain = amgh.Batch([amgh.Problem.from_workload(w) for w in ws]).setup(**amg)
    coop = amgh.Batch([amgh.Problem.from_workload(w) for w in ws]).setup(persistent_cg=1, fuse_coarse=2, **amg)
    u0, _, s0 = plain.solve(yds, **sopts)
    u1, _, s1 = coop.solve(yds, **sopts)
    assert s0 == 0 and s1 == 0
    for a, b in zip(u0, u1):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
