"""Write the frozen expected values under tests/golden/ from the FP64 oracle only.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import aggregate_csr  # noqa: E402


def laplace5x5():
    N = 5
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    A = (sp.kron(I, T) + sp.kron(T, I)).tocsr()
    agg, roots, nagg = aggregate_csr(A.indptr, A.indices, A.data, 0.08)
    with open(os.path.join(HERE, "agg_laplace5x5.txt"), "w") as f:
        f.write("# aggregate id per vertex (row-major 5x5 grid), five-point Laplacian,\n")
        f.write("# theta = 0.08, MIS-2 roots by splitmix64 priority; written by make_golden.py\n")
        f.write("# hand-checked: roots pairwise >= 3 apart in the grid graph; each phase-2 vertex\n")
        f.write("# takes the smallest id among its equally weighted phase-1 neighbours\n")
        f.write(f"# roots: {np.flatnonzero(roots).tolist()}  aggregates: {nagg}\n")
        for r in range(N):
            f.write(" ".join(str(int(a)) for a in agg[r * N:(r + 1) * N]) + "\n")


if __name__ == "__main__":
    laplace5x5()
