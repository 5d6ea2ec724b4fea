"""The bounded device-side waits and round caps, driven to run out on purpose.

Nothing here faults, traps or hangs: amgh_debug_limits only lowers the
limits of waits that are bounded anyway.  With the level-0 staged smoother's
first poll limit at 0, every block of that kernel gives up at once, lets its
bulk copies drain under the separate drain limit, computes nothing and raises
the timeout flag; the call must return AMGH_ERR_TIMEOUT (whatever else its
broken preconditioner did), and once the limit is restored the next call on
the same problem must give the clean result bit for bit.  The aggregation's
distance-2 independent-set loop is capped the same way from the host.
"""
import numpy as np
import pytest

from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TIMEOUT = -8


def test_staged_copy_timeout_is_reported_then_recovers():
    import torch
    from paper_2001_11533_gb300 import amgh
    w = W.unit_square(129, beta=1e-2, jitter=0.2, cfg=141)
    prob = amgh.Problem.from_workload(w).amg_setup(precision=2, coarse_max=64)
    prob.set_solve_opts(inner_tol=1e-10, mass_tol=1e-10, precond_tol=1e-10, inner_max_iter=60)
    u = torch.from_numpy(np.random.default_rng(3).standard_normal(prob.sizes["n"])).cuda()
    clean = prob.hessian_apply(u).cpu().numpy()
    try:
        amgh.debug_limits(bulk_first_polls=0)
        with pytest.raises(amgh.AmghError) as e:
            prob.hessian_apply(u)
        assert e.value.code == TIMEOUT
        with pytest.raises(amgh.AmghError) as e:   # raised again on the next call, and reported again
            prob.hessian_apply(u)
        assert e.value.code == TIMEOUT
    finally:
        amgh.debug_limits(-1, -1)
    again = prob.hessian_apply(u).cpu().numpy()
    assert np.array_equal(again, clean)
    prob.close()


def test_mis_round_cap_is_reported_then_recovers():
    from paper_2001_11533_gb300 import amgh
    w = W.unit_square(65, jitter=0.2, cfg=142)
    ref = amgh.Problem.from_workload(w).amg_setup(coarse_max=32)
    agg_ref, nagg_ref = ref.aggregates(0, 0)
    prob = amgh.Problem.from_workload(w)
    try:
        amgh.debug_limits(mis_round_cap=1)
        with pytest.raises(amgh.AmghError) as e:
            prob.amg_setup(coarse_max=32)
        assert e.value.code == TIMEOUT
    finally:
        amgh.debug_limits(-1, -1)
    prob.amg_setup(coarse_max=32)
    agg, nagg = prob.aggregates(0, 0)
    assert nagg == nagg_ref and np.array_equal(agg, agg_ref)
    prob.close()
    ref.close()


def test_debug_limits_rejects_bad_values():
    from paper_2001_11533_gb300 import amgh
    with pytest.raises(amgh.AmghError) as e:
        amgh.debug_limits(-2, -1)
    assert e.value.code == -1
