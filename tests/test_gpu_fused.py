"""The fused coarse end of the FP32 V-cycle -- one cluster launch for every
level of at most 32768 rows (fuse_coarse 1), or one cooperative launch over
every SM with a bounded software grid barrier for every level of at most
262144 rows (fuse_coarse 2) -- gives the same bits as the level-by-level
kernels, in fewer launches."""
import numpy as np
import pytest

from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("N,precision", [(65, 2), (257, 2), (257, 1)])
def test_fused_equals_level_by_level(N, precision, mode):
    from paper_2001_11533_gb300 import amgh
    w = W.lshape_checkerboard(N=N)
    probs = {}
    for fuse in (mode, 0):
        probs[fuse] = amgh.Problem.from_workload(w).amg_setup(coarse_max=32, precision=precision,
                                                              fuse_coarse=fuse)
    probs[1] = probs.pop(mode)
    sizes = probs[1].query_sizes()
    assert sizes["Ls"] >= 3
    rng = np.random.default_rng(N + precision)
    for lvl in range(sizes["Ls"] - 1):
        f = cuda(rng.standard_normal(sizes["state"][lvl]))
        ya, ia = probs[1].state_solve_level(lvl, f, 1e-10)
        yb, ib = probs[0].state_solve_level(lvl, f, 1e-10)
        assert ia == ib
        assert np.array_equal(ya.cpu().numpy(), yb.cpu().numpy())
    counts = {}
    res = {}
    for fuse, p in probs.items():
        n0 = amgh.launch_count()
        u, _, info = p.solve(tol=1e-10, want_y=False)
        counts[fuse] = amgh.launch_count() - n0
        res[fuse] = (u.cpu().numpy(), info["outer_iters"], info["inner_iters"])
    assert np.array_equal(res[1][0], res[0][0])
    assert res[1][1:] == res[0][1:]
    # the fused path is live on this GPU: the same solve in fewer launches
    assert counts[1] < counts[0]


def test_grid_fused_shared_handle_and_full_size():
    """A handle made by amgh_problem_share runs the level-by-level kernels (the
    batch runtime runs such handles concurrently) and still gives the same
    bits; on the 1025^2 L-shape the grid scope starts at level 1 (107,500
    rows) and the solve matches the level-by-level one bit for bit."""
    from paper_2001_11533_gb300 import amgh
    w = W.lshape_checkerboard(N=1025)
    pa = amgh.Problem.from_workload(w).amg_setup(coarse_max=1000, precision=2, fuse_coarse=2)
    pb = amgh.Problem.from_workload(w).amg_setup(coarse_max=1000, precision=2, fuse_coarse=0)
    sh = pa.share()
    out = []
    for p in (pa, pb, sh):
        n0 = amgh.launch_count()
        u, _, info = p.solve(tol=1e-8, inner_tol=1e-10, mass_tol=1e-8, precond_tol=1e-8, want_y=False)
        out.append((u.cpu().numpy(), info["inner_iters"], amgh.launch_count() - n0))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    assert np.array_equal(out[2][0], out[1][0])
    assert out[0][2] < out[1][2] and out[2][2] == out[1][2]
    sh.close()
    pa.close()
    pb.close()
