"""Batching pattern: independent problems of uneven size with several desired
states each, solved concurrently by the native batch runtime.  Every batched
column must equal the same problem solved alone (same kernels, same order),
and a failing problem must not disturb the others."""
import numpy as np
import pytest

from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _small_batch():
    return W.batch_squares(sizes=(33, 65), per_size=2, rhs=3)


def test_batch_equals_single_problem_solves():
    from paper_2001_11533_gb300 import amgh
    ws = _small_batch()
    opts = dict(coarse_max=600, precision=2)
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(**opts)
    us, infos, st = batch.solve([_cuda(w.y_d) for w in ws], tol=1e-10)
    batch.close()
    assert st == 0 and all(i["status"] == 0 for i in infos)
    for w, u in zip(ws, us):
        single = amgh.Problem.from_workload(w).amg_setup(**opts)
        for c in range(w.y_d.shape[0]):
            single.set_yd(_cuda(w.y_d[c]))
            uc, _, info = single.solve(tol=1e-10)
            assert np.array_equal(uc.cpu().numpy(), u[c].cpu().numpy())


def test_workers_do_not_change_results():
    from paper_2001_11533_gb300 import amgh
    ws = _small_batch()[:2]
    res = []
    for workers in (0, 1, 2):
        probs = [amgh.Problem.from_workload(w) for w in ws]
        batch = amgh.Batch(probs, workers=workers).setup(coarse_max=600)
        us, infos, st = batch.solve([_cuda(w.y_d) for w in ws], tol=1e-10)
        batch.close()
        assert st == 0
        res.append([u.cpu().numpy() for u in us])
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_batch_with_an_empty_column_set():
    """A problem with no desired states is skipped; the others solve."""
    from paper_2001_11533_gb300 import amgh
    import torch
    ws = _small_batch()[:2]
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(coarse_max=600)
    yds = [_cuda(ws[0].y_d), torch.empty((0, ws[1].n_vertices), dtype=torch.float64, device="cuda")]
    us, infos, st = batch.solve(yds, tol=1e-10)
    batch.close()
    assert st == 0 and infos[1]["outer_iters"] == 0 and us[1].shape[0] == 0
    assert infos[0]["outer_iters"] > 0


def test_shared_handle():
    from paper_2001_11533_gb300 import amgh
    w = _small_batch()[0]
    p = amgh.Problem.from_workload(w)
    with pytest.raises(amgh.AmghError):
        p.share()                                   # not set up yet
    p.amg_setup(coarse_max=600)
    q = p.share()
    with pytest.raises(amgh.AmghError):
        q.amg_setup()                               # hierarchy belongs to p
    for h in (p, q):
        h.set_yd(_cuda(w.y_d[1]))
    up, _, ip = p.solve(tol=1e-10)
    uq, _, iq = q.solve(tol=1e-10)
    assert np.array_equal(up.cpu().numpy(), uq.cpu().numpy())
    assert ip["outer_iters"] == iq["outer_iters"]
    q.close()
    # the parent is untouched by its shared handle's life
    up2, _, _ = p.solve(tol=1e-10)
    assert np.array_equal(up.cpu().numpy(), up2.cpu().numpy())


def test_batch_isolates_a_failing_problem():
    from paper_2001_11533_gb300 import amgh
    ws = _small_batch()
    yds = [w.y_d.copy() for w in ws]
    yds[1][2, 33 * 16 + 16] = np.nan        # an interior vertex of the 33^2 grid
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(coarse_max=600)
    us, infos, st = batch.solve([_cuda(y) for y in yds], raise_on_error=False, tol=1e-10)
    batch.close()
    assert st == -7
    assert infos[1]["status"] == -7
    assert all(infos[i]["status"] == 0 for i in (0, 2, 3))


@pytest.mark.slow
def test_full_batch_16_problems_128_rhs():
    """16 jittered squares (65^2 .. 513^2), 8 desired states each, beta log-uniform
    in [1e-6, 1e-2]: all 128 solves reach 1e-8.  The smallest betas need fewer
    Hessian levels (level fallback) and the coarsest level by CG."""
    from paper_2001_11533_gb300 import amgh
    ws = W.batch_squares()
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(coarse_max=1000, precision=2, coarse_solve=1)
    us, infos, st = batch.solve([_cuda(w.y_d) for w in ws], tol=1e-8, precond_tol=1e-8, mass_tol=1e-8,
                                level_fallback=1)
    batch.close()
    assert st == 0
    assert sum(i["outer_iters"] for i in infos) > 0
    assert all(i["final_relres"] <= 1.5e-8 for i in infos)


def test_batch_autotune_keeps_a_candidate_and_the_method():
    """The block-width / slot autotuner times its four candidates, keeps one, and
    the batch then still solves every desired state to the same controls (the
    candidates run the same method per column)."""
    import torch
    from paper_2001_11533_gb300 import amgh
    ws = W.batch_squares(sizes=(33, 65), per_size=1, rhs=4)
    yds = [torch.from_numpy(np.ascontiguousarray(w.y_d)).cuda() for w in ws]
    probs = [amgh.Problem.from_workload(w) for w in ws]
    batch = amgh.Batch(probs).setup(coarse_max=64, precision=2)
    sopts = dict(tol=1e-10, inner_tol=1e-12, mass_tol=1e-12, precond_tol=1e-12)
    ref, _, _ = batch.solve(yds, **sopts)
    choice, times = batch.autotune(yds, **sopts)
    assert choice in amgh.Batch.CANDIDATES and len(times) == 4 and all(t > 0 for t in times.values())
    assert times[choice] == min(times.values())
    us, infos, st = batch.solve(yds, **sopts)
    assert st == 0
    for a, b in zip(us, ref):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        for c in range(a.shape[0]):
            assert np.linalg.norm(a[c] - b[c]) <= 1e-8 * np.linalg.norm(b[c])
    batch.close()
    for p in probs:
        p.close()
