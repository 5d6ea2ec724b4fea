"""The allocation-free aggregation entry point against the regular setup.

For callers that cannot allocate device memory, amgh_aggregate_noalloc runs
the aggregation on a matrix they already hold, with its scratch in a fixed
buffer inside the library.  Its result must be exactly the level-0
aggregates that amgh_amg_setup computes, on consecutive calls (the buffer
keeps the previous call's contents, which must not leak into the next), and
oversized inputs must be rejected.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2001_11533_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup_and_csr(w, hier):
    import torch
    from paper_2001_11533_gb300 import amgh
    prob = amgh.Problem.from_workload(w).amg_setup(coarse_max=32)
    which = "A" if hier == 0 else "KN"
    rp, ci, v, shape = prob.matrix(which, 0)
    ref, nref = prob.aggregates(hier, 0)
    dev = (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(v).cuda())
    return prob, dev, ref, nref


def test_noalloc_matches_setup_on_consecutive_calls():
    import torch
    from paper_2001_11533_gb300 import amgh
    cases = [(W.lshape_checkerboard(N=129), 0),   # 12,033 rows
             (W.unit_square(65, jitter=0.2, cfg=5), 1),  # 4,225 rows, all-vertex stiffness
             (W.lshape_checkerboard(N=129), 1)]   # 12,545 rows
    stream = torch.cuda.current_stream().cuda_stream
    for w, hier in cases + cases[:1]:
        prob, (rp, ci, v), ref, nref = _setup_and_csr(w, hier)
        for _ in range(2):
            out = torch.full((rp.numel() - 1,), -7, dtype=torch.int32, device="cuda")
            nagg = amgh.aggregate_noalloc(rp, ci, v, 0.08, out, stream=stream)
            torch.cuda.synchronize()
            assert nagg == nref
            assert np.array_equal(out.cpu().numpy(), ref)
        prob.close()


def test_noalloc_rejects_oversized_input():
    import torch
    from paper_2001_11533_gb300 import amgh
    n = 40000
    rp = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.arange(n, dtype=torch.int32, device="cuda")
    v = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(amgh.AmghError) as e:
        amgh.aggregate_noalloc(rp, ci, v, 0.08, out)
    assert e.value.code == -1


def test_noalloc_rejects_too_many_entries_and_bad_rowptr():
    """Rows within the limit but more stored entries than the scratch holds, and a
    row-pointer array that does not start at 0: both refused before any kernel."""
    import torch
    from paper_2001_11533_gb300 import amgh
    n, per_row = 1000, 300                       # 300,000 entries > 262,144
    rp = torch.arange(n + 1, dtype=torch.int32, device="cuda") * per_row
    ci = torch.arange(per_row, dtype=torch.int32, device="cuda").repeat(n)
    v = torch.ones(n * per_row, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(amgh.AmghError) as e:
        amgh.aggregate_noalloc(rp, ci, v, 0.08, out)
    assert e.value.code == -1
    rp1 = torch.arange(n + 1, dtype=torch.int32, device="cuda") + 1
    ci1 = torch.arange(n + 1, dtype=torch.int32, device="cuda") % n
    v1 = torch.ones(n + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(amgh.AmghError) as e:
        amgh.aggregate_noalloc(rp1, ci1, v1, 0.08, out)
    assert e.value.code == -1
