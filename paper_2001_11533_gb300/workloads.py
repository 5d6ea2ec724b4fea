"""Seeded synthetic inputs for the linear-quadratic elliptic control problem.

This module builds meshes, coefficients and desired states only: vertex
coordinates, element connectivity, Dirichlet flags, a per-element coefficient
kappa, the regularisation beta and a nodal desired state y_d.  It contains none
of the method's arithmetic (no assembly, no solver, no multigrid), so both the
CUDA path and the FP64 oracle consume exactly the same arrays.

Problem statement (Sec. 2, Eq. functionalcont/pdecont): minimise
1/2 ||y - y_d||^2 + beta/2 ||u||^2 subject to -div(kappa grad y) = u, y = 0 on
the boundary, discretised with P1 elements on triangles (2D) or tetrahedra
(3D).  The paper's meshes (a 474-element tet mesh, an engine bracket) are not
available, so the workloads below are synthetic stand-ins with the shapes,
sizes and coefficient structure of the paper's experiments (Sec. 5.3-5.6).

Conventions (readings of points the paper leaves open):
  * structured 2D grid of N x N vertices on [0,1]^2, vertex id = i + N*j;
    each square (i,j) is split along the diagonal (i,j)-(i+1,j+1) into the
    lower triangle (v00, v10, v11) followed by the upper one (v00, v11, v01);
    elements are ordered square-major;
  * structured 3D grid of N^3 vertices, vertex id = i + N*j + N^2*k; each cube
    is split into the 6 Kuhn tetrahedra 0 -> e_a -> e_a + e_b -> (1,1,1) over
    the permutations (a, b, c) of (x, y, z) in lexicographic order;
  * boundary vertices are those on a boundary edge (2D) / face (3D), i.e. an
    edge/face that belongs to exactly one element; all boundary vertices are
    Dirichlet (y = 0) unless stated otherwise;
  * every random draw uses numpy.random.default_rng(SeedSequence([cfg, stream])).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One control problem instance (host arrays, ready for both sides)."""

    name: str
    dim: int
    coords: np.ndarray          # (n, dim) float64
    elements: np.ndarray        # (ne, dim+1) int32, 0-based vertex ids
    dirichlet: np.ndarray       # (n,) uint8, 1 = Dirichlet vertex (y = 0)
    kappa: np.ndarray           # (ne,) float64, per element
    beta: float
    y_d: np.ndarray             # (n,) float64 nodal desired state (or (k, n) for batches)
    meta: dict = field(default_factory=dict)

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elements(self) -> int:
        return int(self.elements.shape[0])

    @property
    def n_interior(self) -> int:
        return int(self.n_vertices - int(self.dirichlet.sum()))


def _rng(cfg: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([cfg, stream]))


# --------------------------------------------------------------------------- meshes

def grid2d(N: int):
    """N x N vertex grid on [0,1]^2 split into 2 (N-1)^2 triangles."""
    h = 1.0 / (N - 1)
    i = np.arange(N)
    X, Y = np.meshgrid(i * h, i * h, indexing="xy")  # X[j, i] = i*h
    coords = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    ii, jj = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    v00 = ii + N * jj
    v10 = v00 + 1
    v01 = v00 + N
    v11 = v00 + N + 1
    lower = np.stack([v00, v10, v11], axis=1)
    upper = np.stack([v00, v11, v01], axis=1)
    elems = np.empty((2 * lower.shape[0], 3), dtype=np.int64)
    elems[0::2] = lower
    elems[1::2] = upper
    return coords, elems.astype(np.int32)


def grid3d_kuhn(N: int):
    """N^3 vertex grid on [0,1]^3 split into 6 (N-1)^3 Kuhn tetrahedra."""
    h = 1.0 / (N - 1)
    i = np.arange(N, dtype=np.float64) * h
    K, J, I = np.meshgrid(i, i, i, indexing="ij")  # I fastest
    coords = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    del K, J, I
    it = np.int64 if N ** 3 >= 2 ** 31 else np.int32
    c = np.arange(N - 1, dtype=it)
    CK, CJ, CI = np.meshgrid(c, c, c, indexing="ij")
    base = (CI + N * CJ + N * N * CK).ravel()
    del CK, CJ, CI
    step = {0: 1, 1: N, 2: N * N}
    elems = np.empty((base.size, 6, 4), dtype=np.int32)  # cube-major, 6 per cube
    for t, perm in enumerate(itertools.permutations((0, 1, 2))):
        a, b, _ = perm
        elems[:, t, 0] = base
        elems[:, t, 1] = base + step[a]
        elems[:, t, 2] = base + step[a] + step[b]
        elems[:, t, 3] = base + 1 + N + N * N
    return coords, elems.reshape(-1, 4)


def cube_boundary(N: int) -> np.ndarray:
    """Boundary flags of the N^3 structured grid (same set as boundary_vertices)."""
    i = np.arange(N)
    on = (i == 0) | (i == N - 1)
    K, J, I = np.meshgrid(on, on, on, indexing="ij")
    return (K | J | I).ravel().astype(np.uint8)


def boundary_vertices(elements: np.ndarray, n: int) -> np.ndarray:
    """Flag vertices on a facet that belongs to exactly one element."""
    d1 = elements.shape[1]
    facets = []
    for drop in range(d1):
        keep = [k for k in range(d1) if k != drop]
        facets.append(elements[:, keep])
    F = np.sort(np.concatenate(facets, axis=0).astype(np.int64), axis=1)
    # encode facet as a single int64 key (vertex ids < 2^21 per slot for 3D)
    if d1 == 3:
        key = F[:, 0] * (n + 1) + F[:, 1]
    else:
        key = (F[:, 0] * (n + 1) + F[:, 1]) * (n + 1) + F[:, 2]
    uniq, counts = np.unique(key, return_counts=True)
    single = np.isin(key, uniq[counts == 1])
    flags = np.zeros(n, dtype=np.uint8)
    flags[F[single].ravel()] = 1
    return flags


def remove_vertices(coords, elems, keep_mask):
    """Drop elements touching a removed vertex and renumber the rest (ascending id)."""
    ok = keep_mask[elems].all(axis=1)
    elems = elems[ok]
    newid = -np.ones(coords.shape[0], dtype=np.int64)
    newid[keep_mask] = np.arange(int(keep_mask.sum()))
    return coords[keep_mask].copy(), newid[elems].astype(np.int32)


def element_measure(coords, elems):
    """Signed-free element size (area/volume) used only to validate generated meshes."""
    d = coords.shape[1]
    P = coords[elems]
    E = P[:, 1:, :] - P[:, :1, :]
    det = np.linalg.det(E) if d == 3 else E[:, 0, 0] * E[:, 1, 1] - E[:, 0, 1] * E[:, 1, 0]
    return np.abs(det) / math.factorial(d)


def jitter_interior(coords, dirichlet, h, frac, rng):
    """Move non-boundary vertices by independent U[-frac h, frac h] per coordinate."""
    c = coords.copy()
    move = dirichlet == 0
    c[move] += rng.uniform(-frac * h, frac * h, size=(int(move.sum()), coords.shape[1]))
    return c


def centroids(coords, elems):
    """Element centroids, one vertex gather at a time (no (ne, d+1, d) temporary)."""
    out = coords[elems[:, 0]].copy()
    for k in range(1, elems.shape[1]):
        out += coords[elems[:, k]]
    out /= elems.shape[1]
    return out


def gaussian_bumps(x, centres, amps, width):
    """Sum_k a_k exp(-|x - c_k|^2 / (2 width^2)) evaluated at the rows of x."""
    out = np.zeros(x.shape[0])
    for c, a in zip(centres, amps):
        r2 = ((x - c[None, :]) ** 2).sum(axis=1)
        out += a * np.exp(-r2 / (2.0 * width * width))
    return out


def gaussian_bumps_grid3(N, centres, amps, width):
    """gaussian_bumps at the vertices of the N^3 grid of grid3d_kuhn (x fastest),
    using exp(-|x - c|^2 / 2w^2) = prod over axes of exp(-(x_a - c_a)^2 / 2w^2):
    the same function up to rounding, without a (vertices x bumps) pass of exp."""
    t = np.arange(N, dtype=np.float64) * (1.0 / (N - 1))
    e = [np.exp(-((t[None, :] - centres[:, a:a + 1]) ** 2) / (2.0 * width * width)) for a in range(3)]
    zy = (amps[:, None, None] * e[2][:, :, None] * e[1][:, None, :]).reshape(len(amps), N * N)
    return (zy.T @ e[0]).ravel()


def _bump_params(rng, k, dim, inside):
    centres = []
    while len(centres) < k:
        p = rng.uniform(0.0, 1.0, size=dim)
        if inside(p):
            centres.append(p)
    amps = rng.uniform(-1.0, 1.0, size=k)
    return np.array(centres), amps


# --------------------------------------------------------------------------- configs

def unit_square(N: int, beta: float = 1e-2, y_d: str = "sin", cfg: int = 0,
                jitter: float = 0.0, stream: int = 1, name: str | None = None) -> Workload:
    """Unit square, N x N grid, kappa = 1.

    y_d = "sin": sin(pi x) sin(pi y) (the tiny FP64 case);
    y_d = "exact": (1/(2 pi^2) + 2 pi^2 beta) sin sin, the 2D analogue of the
    paper's closed-form test state (Sec. 5.3, Eq. test-state), whose optimal
    control is u* = sin(pi x) sin(pi y).
    """
    coords, elems = grid2d(N)
    dirichlet = boundary_vertices(elems, coords.shape[0])
    if jitter > 0.0:
        coords = jitter_interior(coords, dirichlet, 1.0 / (N - 1), jitter, _rng(cfg, stream))
    x, y = coords[:, 0], coords[:, 1]
    s = np.sin(np.pi * x) * np.sin(np.pi * y)
    if y_d == "sin":
        yd = s
    elif y_d == "exact":
        yd = (1.0 / (2.0 * np.pi ** 2) + 2.0 * np.pi ** 2 * beta) * s
    else:
        raise ValueError(y_d)
    return Workload(name or f"square{N}", 2, coords, elems, dirichlet,
                    np.ones(elems.shape[0]), float(beta), yd,
                    {"N": N})


def tiny_fp64() -> Workload:
    """33 x 33 unit square, kappa = 1, beta = 1e-2, y_d = sin sin, 3 AMG levels."""
    w = unit_square(33, beta=1e-2, y_d="sin", name="square33_fp64")
    w.meta.update({"levels": 3, "tol": 1e-10})
    return w


def lshape_checkerboard(N: int = 1025, cfg: int = 1) -> Workload:
    """L-shaped domain [0,1]^2 minus (0.5,1]^2 from an N x N grid.

    Interior vertices jittered by U[-0.2h, 0.2h] (stream 1); kappa on an 8x8
    checkerboard over [0,1]^2, each cell 1 or 1e4 with probability 1/2
    (stream 2), evaluated at the element centroid; beta = 1e-4; y_d a sum of
    8 Gaussian bumps of width (standard deviation) 0.1 with centres uniform in
    the L and amplitudes U[-1,1] (stream 3).
    """
    assert (N - 1) % 2 == 0
    coords, elems = grid2d(N)
    mid = (N - 1) // 2
    idx = np.arange(N * N)
    i, j = idx % N, idx // N
    keep = ~((i > mid) & (j > mid))
    coords, elems = remove_vertices(coords, elems, keep)
    n = coords.shape[0]
    dirichlet = boundary_vertices(elems, n)
    h = 1.0 / (N - 1)
    coords = jitter_interior(coords, dirichlet, h, 0.2, _rng(cfg, 1))
    vol = element_measure(coords, elems)
    assert (vol > 0).all(), "jitter produced a degenerate element"
    cells = _rng(cfg, 2).random(64) < 0.5
    vals = np.where(cells, 1e4, 1.0).reshape(8, 8)   # [cy, cx]
    c = centroids(coords, elems)
    cx = np.minimum((c[:, 0] * 8).astype(np.int64), 7)
    cy = np.minimum((c[:, 1] * 8).astype(np.int64), 7)
    kappa = vals[cy, cx].astype(np.float64)
    inside_l = lambda p: not (p[0] > 0.5 and p[1] > 0.5)
    cen, amps = _bump_params(_rng(cfg, 3), 8, 2, inside_l)
    yd = gaussian_bumps(coords, cen, amps, 0.1)
    return Workload(f"lshape{N}_checker", 2, coords, elems, dirichlet, kappa, 1e-4, yd,
                    {"N": N, "grid": f"{N}x{N} L-shape"})


def cube_grf(N: int = 129, cfg: int = 2, features: int = 1024, corr: float = 0.1) -> Workload:
    """Unit cube, N^3 grid, Kuhn tets; kappa = exp(g), g a Gaussian random field.

    g has unit variance and squared-exponential covariance of length `corr`,
    sampled by `features` random Fourier features (stream 4) at tet centroids;
    beta = 1e-5; y_d from 8 Gaussian bumps of width 0.1 (stream 3).
    """
    coords, elems = grid3d_kuhn(N)
    dirichlet = cube_boundary(N)
    rng = _rng(cfg, 4)
    omega = rng.normal(0.0, 1.0 / corr, size=(features, 3))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=features)
    c = centroids(coords, elems)
    g = np.zeros(elems.shape[0])
    scale = math.sqrt(2.0 / features)
    chunk = 1 << 18
    for s in range(0, c.shape[0], chunk):
        g[s:s + chunk] = scale * np.cos(c[s:s + chunk] @ omega.T + phase[None, :]).sum(axis=1)
    kappa = np.exp(g)
    cen, amps = _bump_params(_rng(cfg, 3), 8, 3, lambda p: True)
    yd = gaussian_bumps(coords, cen, amps, 0.1)
    return Workload(f"cube{N}_grf", 3, coords, elems, dirichlet, kappa, 1e-5, yd, {"N": N})


def batch_squares(cfg: int = 3, sizes=(65, 129, 257, 513), per_size: int = 4, rhs: int = 8):
    """Independent jittered unit squares with several desired states each.

    Jitter U[-0.2h, 0.2h] (stream 10+p); kappa = 1; beta_p = 10^U[-6,-2]
    (stream 7); `rhs` desired states per problem from the 8-bump recipe
    (stream 20+p).
    """
    betas = 10.0 ** _rng(cfg, 7).uniform(-6.0, -2.0, size=len(sizes) * per_size)
    out = []
    p = 0
    for N in sizes:
        for _ in range(per_size):
            coords, elems = grid2d(N)
            dirichlet = boundary_vertices(elems, coords.shape[0])
            coords = jitter_interior(coords, dirichlet, 1.0 / (N - 1), 0.2, _rng(cfg, 10 + p))
            rng = _rng(cfg, 20 + p)
            yds = []
            for _k in range(rhs):
                cen, amps = _bump_params(rng, 8, 2, lambda q: True)
                yds.append(gaussian_bumps(coords, cen, amps, 0.1))
            out.append(Workload(f"batch{p}_sq{N}", 2, coords, elems, dirichlet,
                                np.ones(elems.shape[0]), float(betas[p]), np.stack(yds), {"N": N}))
            p += 1
    return out


def cube_slabs(N: int = 257, cfg: int = 4) -> Workload:
    """Unit cube, N^3 Kuhn grid, kappa alternating 1 / 1e6 in 10 slabs along x3.

    Slab boundaries k/10 jittered by U[-0.02, 0.02] (stream 8) and sorted;
    beta = 1e-6; y_d from 32 Gaussian bumps of width 0.05 (stream 9).
    """
    coords, elems = grid3d_kuhn(N)
    dirichlet = cube_boundary(N)
    bnd = np.sort(np.arange(1, 10) / 10.0 + _rng(cfg, 8).uniform(-0.02, 0.02, size=9))
    # x3 of an element centroid (the same sums as centroids()) depends only on
    # the cube's layer and on which of the 6 Kuhn tets it is: tabulate it from
    # the first column of cubes and repeat it over each layer
    x3 = coords[:, 2]
    col = elems.reshape(N - 1, (N - 1) ** 2, 6, 4)[:, 0]          # (layer, tet, vertex)
    z = x3[col[:, :, 0]]
    for k in range(1, 4):
        z = z + x3[col[:, :, k]]
    z = z / 4.0
    kap = np.where(np.searchsorted(bnd, z) % 2 == 0, 1.0, 1e6)    # (layer, tet)
    kappa = np.broadcast_to(kap[:, None, :], (N - 1, (N - 1) ** 2, 6)).reshape(-1).copy()
    cen, amps = _bump_params(_rng(cfg, 9), 32, 3, lambda p: True)
    yd = gaussian_bumps_grid3(N, cen, amps, 0.05)
    return Workload(f"cube{N}_slabs", 3, coords, elems, dirichlet, kappa, 1e-6, yd, {"N": N})


def cube_ball(N: int = 33, contrast: float = 1e-2, cfg: int = 5) -> Workload:
    """The varying-coefficient setting of Sec. 5.6 (Table 7) on an N^3 Kuhn grid:
    kappa = contrast inside the ball |x - (1/2,1/2,1/2)| <= 1/4 (element centroid)
    and 1 outside, so the mesh does not follow the coefficient; zero Dirichlet
    condition on the face x3 = 0 only (homogeneous Neumann elsewhere); desired
    state y_d = 1; beta = 1.  Unjittered, so cfg is unused."""
    coords, elems = grid3d_kuhn(N)
    dirichlet = (np.abs(coords[:, 2]) < 0.5 / (N - 1)).astype(np.uint8)
    c = centroids(coords, elems)
    inside = ((c - 0.5) ** 2).sum(axis=1) <= 0.25 ** 2
    kappa = np.where(inside, float(contrast), 1.0)
    yd = np.ones(coords.shape[0])
    return Workload(f"cube{N}_ball{contrast:g}", 3, coords, elems, dirichlet, kappa, 1.0, yd,
                    {"N": N, "contrast": contrast})


def random_vectors(n: int, k: int, cfg: int, stream: int) -> np.ndarray:
    """Seeded standard normal test vectors, shape (k, n)."""
    return _rng(cfg, stream).standard_normal((k, n))
