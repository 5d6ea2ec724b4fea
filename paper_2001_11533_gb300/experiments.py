"""The paper's experiments on this GPU path, at the sizes of its tables.

Each function runs the CUDA library through its C ABI on seeded synthetic
inputs and returns plain rows; nothing here computes any of the method.

  a_numbers_table   Sec. 5.1, Tables 1-2: a_j (Eq. ajnumerical) and a~_j
                    (Eq. aj-tilde) by the power method, for the geometric
                    hierarchy and for AMG with and without aggressive
                    first-level coarsening, with the ratios a_j / a_j+1.
  two_grid_table    Sec. 5.4, Table 5: two-grid outer CG counts of the AMG and
                    the geometric hierarchy on structured squares (the
                    table's N are 2D vertex counts, so the 2D setting).
  level_sweep_table Sec. 5.6, Table 7: outer CG counts and times for the
                    ball-inclusion cube (Dirichlet on x3 = 0 only) with no
                    preconditioner and with 2..5 Hessian levels.
"""
from __future__ import annotations

import time

import numpy as np

from . import amgh, workloads


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def a_numbers_table(N: int = 65, levels: int = 3, iters: int = 60, tol: float = 1e-12):
    rows = {}
    w = workloads.unit_square(N)
    kinds = {"geometric": dict(geometric=1, coarse_max=1), "amg_aggressive": dict(aggressive=1, coarse_max=8),
             "amg": dict(coarse_max=8)}
    for kind, opts in kinds.items():
        p = amgh.Problem.from_workload(w).amg_setup(**opts)
        p.set_solve_opts(inner_tol=tol, mass_tol=tol)
        L = min(p.sizes["Ls"], p.sizes["Lc"])
        out = []
        for j in range(min(levels + 1, L - 1)):
            v0 = _cuda(np.random.default_rng(100 + j).standard_normal(p.sizes["control"][j]))
            out.append({"level": j, "a": p.aj_estimate(j, v0, weighted=True, iters=iters),
                        "a_tilde": p.aj_estimate(j, v0, weighted=False, iters=iters),
                        "controls": p.sizes["control"][j]})
        for j in range(1, len(out)):
            out[j]["ratio_a_prev_over_a"] = out[j - 1]["a"] / out[j]["a"]
        rows[kind] = out
        p.close()
    return {"mesh": f"unit square {N}^2, P1 triangles, kappa = 1", "power_iterations": iters, "rows": rows}


def two_grid_table(sizes=(9, 17, 33, 65, 129, 257), betas=(1e-4, 1e-6), tol=1e-8):
    rows = []
    for N in sizes:
        row = {"N": N * N}
        for beta in betas:
            w = workloads.unit_square(N, beta=beta, y_d="exact")
            for kind, opts in (("amg", dict(coarse_max=1)), ("geometric", dict(geometric=1, coarse_max=1))):
                p = amgh.Problem.from_workload(w).amg_setup(hessian_levels=2, coarse_solve=2, **opts)
                _, _, info = p.solve(tol=tol, inner_tol=1e-10, mass_tol=1e-10, precond_tol=1e-10, coarse_tol=1e-10,
                                     want_y=False, raise_on_error=False)
                row[f"{kind}_beta{beta:g}"] = info["outer_iters"] if info["status"] == 0 else f"status {info['status']}"
                p.close()
        rows.append(row)
    return {"setting": "unit square, P1 triangles, kappa = 1, y_d of the closed-form optimum; two-grid "
                       "(hessian_levels 2), coarse Hessian dense up to 4096 controls else CG to 1e-10",
            "rows": rows}


def level_sweep_table(N: int = 65, contrasts=(1e-4, 1e-3, 1e-2, 1e-1, 1.0), levels=(0, 2, 3, 4, 5),
                      tol: float = 1e-8, precision: int = 2):
    import torch
    rows = []
    for c in contrasts:
        w = workloads.cube_ball(N=N, contrast=c)
        row = {"contrast": c}
        for L in levels:
            p = amgh.Problem.from_workload(w).amg_setup(precision=precision, coarse_max=16,
                                                         hessian_levels=max(L, 2), coarse_solve=2)
            if L and min(p.sizes["Ls"], p.sizes["Lc"]) < L:
                row[str(L)] = "fewer levels"
                p.close()
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, info = p.solve(tol=tol, precond=1 if L else 0, inner_tol=1e-10, mass_tol=1e-8, precond_tol=1e-8,
                                 want_y=False, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            key = str(L) if L else "none"
            row[key] = {"outer": info["outer_iters"], "s": round(dt, 3)} if info["status"] == 0 else \
                {"status": info["status"], "outer": info["outer_iters"]}
            p.close()
        rows.append(row)
    return {"setting": f"{N}^3 Kuhn cube, kappa = contrast in the ball |x - c| <= 1/4, Dirichlet on x3 = 0 only, "
                       f"y_d = 1, beta = 1, precision {precision}", "rows": rows}
