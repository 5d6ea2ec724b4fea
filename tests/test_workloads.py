"""Checks of the seeded input generators (no method arithmetic involved)."""
import numpy as np

from paper_2001_11533_gb300 import workloads as W


def test_sizes_of_the_configs():
    w = W.tiny_fp64()
    assert (w.n_vertices, w.n_interior, w.n_elements) == (1089, 961, 2048)
    w = W.lshape_checkerboard(N=65)
    assert w.n_vertices == 65 * 65 - 32 * 32
    assert w.n_elements == 2 * (64 * 64 - 32 * 32)
    assert set(np.unique(w.kappa)) <= {1.0, 1e4}
    assert (W.element_measure(w.coords, w.elements) > 0).all()


def test_structured_cube_boundary_matches_generic():
    for N in (3, 5, 8):
        c, e = W.grid3d_kuhn(N)
        assert np.array_equal(W.cube_boundary(N), W.boundary_vertices(e, c.shape[0]))
        assert abs(W.element_measure(c, e).sum() - 1.0) < 1e-12


def test_seeded_reproducible():
    a = W.lshape_checkerboard(N=33)
    b = W.lshape_checkerboard(N=33)
    assert np.array_equal(a.coords, b.coords) and np.array_equal(a.y_d, b.y_d)
    assert np.array_equal(a.kappa, b.kappa)
    c = W.cube_grf(N=5, features=32)
    assert np.all(c.kappa > 0) and c.dim == 3
    batch = W.batch_squares(sizes=(9, 17), per_size=2, rhs=3)
    assert len(batch) == 4 and batch[0].y_d.shape == (3, 81)
    assert all(1e-6 <= p.beta <= 1e-2 for p in batch)


def test_separable_bumps_match_direct_sum():
    N = 9
    coords, _ = W.grid3d_kuhn(N)
    cen, amps = W._bump_params(W._rng(4, 9), 5, 3, lambda p: True)
    a = W.gaussian_bumps(coords, cen, amps, 0.2)
    b = W.gaussian_bumps_grid3(N, cen, amps, 0.2)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-15)


def test_cube_slabs_kappa_from_centroid_height():
    w = W.cube_slabs(N=9)
    z = W.centroids(w.coords, w.elements)[:, 2]
    bnd = np.sort(np.arange(1, 10) / 10.0 + W._rng(4, 8).uniform(-0.02, 0.02, size=9))
    assert np.array_equal(w.kappa, np.where(np.searchsorted(bnd, z) % 2 == 0, 1.0, 1e6))


def test_cube_ball_boundary_and_coefficient():
    w = W.cube_ball(N=9, contrast=1e-3)
    z = w.coords[:, 2]
    assert np.array_equal(w.dirichlet.astype(bool), z == 0.0)
    assert w.n_interior == 9 * 9 * 8
    c = W.centroids(w.coords, w.elements)
    inside = np.linalg.norm(c - 0.5, axis=1) <= 0.25
    assert inside.any() and (~inside).any()
    assert np.array_equal(w.kappa, np.where(inside, 1e-3, 1.0)) and w.beta == 1.0
    assert np.all(w.y_d == 1.0)
