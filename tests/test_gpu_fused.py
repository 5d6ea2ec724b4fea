"""The fused coarse end of the FP32 V-cycle (one cluster launch for every
level of at most 32768 rows) gives the same bits as the level-by-level
kernels, in fewer launches."""
import numpy as np
import pytest

from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("N,precision", [(65, 2), (257, 2), (257, 1)])
def test_fused_equals_level_by_level(N, precision):
    from paper_2001_11533_gb300 import amgh
    w = W.lshape_checkerboard(N=N)
    probs = {}
    for fuse in (1, 0):
        probs[fuse] = amgh.Problem.from_workload(w).amg_setup(coarse_max=32, precision=precision,
                                                              fuse_coarse=fuse)
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
