"""The dense SPD inverse behind the exact coarsest solves (Sec. 3.2), on its own.

amgh_dense_spd_inverse runs the same kernels as the coarsest-level setup
(32-wide panel Cholesky fused with the L^-1 sweep, lookahead, W^T W).  Its
result must be the inverse, which numpy's LU-based inverse defines here, to
within a bound set by the conditioning, at sizes below, on and around the
panel width and up to the 4096-row limit; only the lower triangle may be
read (the upper one is NaN here); a pivot that is not positive must be
reported by its row.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def spd(n, seed, alpha=1e-3):
    """B B^T / n + alpha I: eigenvalues in about [alpha, 4 + alpha]."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((n, n))
    return b @ b.T / n + alpha * np.eye(n)


def gpu_inverse(a):
    import torch
    from paper_2001_11533_gb300 import amgh
    n = a.shape[0]
    lower = np.tril(a) + np.triu(np.full((n, n), np.nan), 1)
    a_dev = torch.from_numpy(lower).cuda()
    keep = a_dev.clone()
    inv = torch.empty_like(a_dev)
    st, info = amgh.dense_spd_inverse(a_dev, inv)
    assert torch.equal(torch.nan_to_num(a_dev, nan=7.0), torch.nan_to_num(keep, nan=7.0))
    return st, info, inv.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 17, 31, 32, 33, 63, 64, 65, 100, 257, 845, 847, 1000, 4096])
def test_inverse_matches_definition(n):
    a = spd(n, seed=n)
    st, info, x = gpu_inverse(a)
    assert st == 0 and info == 0
    ref = np.linalg.inv(a)
    assert np.array_equal(x, x.T)  # the upper triangle is mirrored
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    # cond(a) is at most about 4e3: a backward-stable inverse is accurate to
    # a few times cond * n^(1/2) * eps, far below this bound
    assert err <= 1e-9, err
    assert np.linalg.norm(a @ x - np.eye(n)) / np.sqrt(n) <= 1e-10


def test_inverse_of_a_laplacian_with_a_ragged_panel():
    """The 5-point Laplacian of a 29 x 29 grid (841 rows, last panel 9 wide)."""
    m = 29
    t = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    a = np.kron(t, np.eye(m)) + np.kron(np.eye(m), t)
    st, info, x = gpu_inverse(a)
    assert st == 0
    ref = np.linalg.inv(a)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-11


@pytest.mark.parametrize("n,row,val", [(8, 6, -1.0), (70, 41, 0.0), (70, 64, -3.0), (300, 300, -2.0)])
def test_non_positive_pivot_is_reported(n, row, val):
    """A diagonal matrix's pivots are its entries: the first one that is not
    positive (1-based row) comes back with INDEFINITE."""
    from paper_2001_11533_gb300 import amgh
    d = np.linspace(1.0, 2.0, n)
    d[row - 1] = val
    st, info, _ = gpu_inverse(np.diag(d))
    assert st == amgh.ERR_INDEFINITE and info == row


def test_indefinite_two_by_two_and_limits():
    """[[1, 2], [2, 1]]: the second pivot is 1 - 4 < 0.  n outside 1..4096 is
    refused before any kernel runs."""
    import torch
    from paper_2001_11533_gb300 import amgh
    st, info, _ = gpu_inverse(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert st == amgh.ERR_INDEFINITE and info == 2
    for n in (4097,):
        a = torch.eye(n, dtype=torch.float64, device="cuda")
        with pytest.raises(amgh.AmghError) as e:
            amgh.dense_spd_inverse(a, torch.empty_like(a))
        assert e.value.code == -1


def test_concurrent_inverses_on_several_streams():
    """Eight host threads, each on its own CUDA stream, invert different
    matrices at once (as the batch runtime's solve slots do when each falls
    back to a coarser Hessian level): every result must still be the inverse.
    Contention changes when each block of a launch starts, so a kernel whose
    blocks read data that other blocks of the same launch overwrite fails here."""
    import threading
    import torch
    from paper_2001_11533_gb300 import amgh
    n, jobs = 1000, 8
    mats = [spd(n, seed=100 + j) for j in range(jobs)]
    refs = [np.linalg.inv(a) for a in mats]
    devs = [torch.from_numpy(np.tril(a)).cuda() for a in mats]
    outs = [torch.empty_like(d) for d in devs]
    streams = [torch.cuda.Stream() for _ in range(jobs)]
    torch.cuda.synchronize()
    errors = []

    def work(j):
        try:
            for _ in range(3):
                st, info = amgh.dense_spd_inverse(devs[j], outs[j], stream=streams[j].cuda_stream)
                assert st == 0 and info == 0
                x = outs[j].cpu().numpy()
                err = np.linalg.norm(x - refs[j]) / np.linalg.norm(refs[j])
                assert err <= 1e-9, (j, err)
        except Exception as e:  # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(j,)) for j in range(jobs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors


def test_fp64_peak_is_measured():
    """amgh_fp64_peak: both forms give a positive rate, within a plausible band
    of the part's FP64 rate (GB300: about 1.25 TFLOP/s nominal for either);
    an unknown kind is refused."""
    from paper_2001_11533_gb300 import amgh
    for kind in (0, 1):
        t = amgh.fp64_peak(kind)
        assert 0.1 < t < 200.0, (kind, t)
    with pytest.raises(amgh.AmghError) as e:
        amgh.fp64_peak(2)
    assert e.value.code == -1
