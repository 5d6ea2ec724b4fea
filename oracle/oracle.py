"""Python handle on the FP64 CPU oracle (amgh_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
benchmark's CPU-baseline / reference leg are the only callers.  The oracle
shares no code with the CUDA path; this module only compiles the C file with
gcc (-O2 -ffp-contract=off, no fused multiply-add) and marshals numpy arrays
through ctypes.  A second build with -fopenmp (omp=True) splits the
solve-phase row loops over the host's cores for the benchmark's multi-core
CPU timing; its results are bit-identical to the sequential build.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amgh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libamgh_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libamgh_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

OK, INVALID, NOT_SETUP, OOM, NOT_CONVERGED, INDEFINITE, NUMERIC = 0, -1, -2, -4, -5, -6, -7
MATRIX = {"A": 0, "My": 1, "Myu": 2, "S": 3, "KN": 4, "Mu": 5, "P": 6, "Kfull": 7, "Mfull": 8}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into oracle/_build (idempotent); omp=True: the
    -fopenmp build of the same file."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP if omp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    if omp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def lib(omp: bool = False):
    with _lock:
        if omp not in _libs:
            L = C.CDLL(build(omp=omp))
            P, I, L64, D = C.c_void_p, C.c_int, C.c_long, C.c_double
            sig = {
                "orc_create": [I, L64, P, L64, P, P, P, D, P, P],
                "orc_set_yd": [P, P],
                "orc_setup": [P, I, I, D, I, I, I, I],
                "orc_set_tols": [P, D, D, I, I],
                "orc_set_precond_tol": [P, D],
                "orc_set_hierarchy": [P, I, I],
                "orc_set_coarse_solve": [P, I, D, I, P],
                "orc_sizes": [P, P, P, P, P, P, P, P],
                "orc_matrix_info": [P, I, I, P, P, P],
                "orc_matrix_copy": [P, I, I, P, P, P],
                "orc_aggregates": [P, I, I, P, P],
                "orc_aggregate_csr": [I, P, P, P, D, P, P, P],
                "orc_vcycle": [P, I, P, P],
                "orc_smooth": [P, I, P, P, I],
                "orc_state_solve": [P, I, D, P, P, P],
                "orc_mass_solve": [P, I, P, P, P],
                "orc_hessian": [P, I, P, P],
                "orc_mlas": [P, I, I, P, P],
                "orc_rhs": [P, P],
                "orc_objective": [P, P, P, P, P],
                "orc_solve": [P, I, D, I, P, P, P, P, P],
                "orc_counters": [P, P, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.orc_destroy.argtypes = [P]
            L.orc_destroy.restype = None
            L.orc_priority.argtypes = [C.c_uint64]
            L.orc_priority.restype = C.c_uint64
            L.orc_threads.argtypes = []
            L.orc_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            _libs[omp] = L
    return _libs[omp]


def threads(omp: bool = True) -> int:
    """Threads the row loops of that build use."""
    return int(lib(omp).orc_threads())


def set_threads(t: int) -> int:
    """Threads of the -fopenmp build's row loops; returns the number in effect."""
    lib(True).orc_set_threads(int(t))
    return threads(True)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


def priority(i: int) -> int:
    return int(lib().orc_priority(int(i)))


def aggregate_csr(rp, ci, v, theta):
    """Aggregate an arbitrary symmetric CSR matrix; returns (agg, roots, nagg)."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    n = rp.shape[0] - 1
    agg = np.empty(n, dtype=np.int32)
    roots = np.empty(n, dtype=np.uint8)
    nagg = C.c_int(0)
    _check(lib().orc_aggregate_csr(n, _p(rp), _p(ci), _p(v), float(theta), _p(agg), _p(roots),
                                   C.byref(nagg)), "aggregate_csr")
    return agg, roots.astype(bool), nagg.value


class Oracle:
    """One control problem on the CPU: assembly, AMG hierarchies, solves."""

    def __init__(self, w, max_levels=25, hessian_levels=0, theta=0.08, coarse_max=256,
                 smoother=1, degree=2, smooth_prolongator=1, inner_tol=1e-10, mass_tol=1e-10,
                 inner_maxit=1000, mass_maxit=1000, setup=True, omp=False, aggressive=0, geometric=0):
        self.w = w
        self._L = L = lib(omp)
        self._coords = np.ascontiguousarray(w.coords, dtype=np.float64)
        self._elems = np.ascontiguousarray(w.elements, dtype=np.int32)
        self._dir = np.ascontiguousarray(w.dirichlet, dtype=np.uint8)
        self._kappa = np.ascontiguousarray(w.kappa, dtype=np.float64)
        yd = w.y_d if w.y_d.ndim == 1 else w.y_d[0]
        self._yd = np.ascontiguousarray(yd, dtype=np.float64)
        h = C.c_void_p()
        _check(L.orc_create(w.dim, w.n_vertices, _p(self._coords), w.n_elements, _p(self._elems),
                            _p(self._dir), _p(self._kappa), float(w.beta), _p(self._yd),
                            C.byref(h)), "create")
        self.h = h
        self.m = int(w.n_interior)
        self.n = int(w.n_vertices)
        _check(L.orc_set_hierarchy(self.h, int(aggressive), int(geometric)), "set_hierarchy")
        if setup:
            self.setup(max_levels, hessian_levels, theta, coarse_max, smoother, degree,
                       smooth_prolongator)
            self.set_tols(inner_tol, mass_tol, inner_maxit, mass_maxit)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._L.orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # -- setup / queries
    def setup(self, max_levels=25, hessian_levels=0, theta=0.08, coarse_max=256, smoother=1,
              degree=2, smooth_prolongator=1):
        _check(self._L.orc_setup(self.h, max_levels, hessian_levels, theta, coarse_max, smoother,
                               degree, smooth_prolongator), "setup")
        self.set_tols(1e-10, 1e-10, 1000, 1000)

    def set_tols(self, inner_tol, mass_tol, inner_maxit=1000, mass_maxit=1000):
        _check(self._L.orc_set_tols(self.h, inner_tol, mass_tol, inner_maxit, mass_maxit), "tols")

    def set_precond_tol(self, pc_inner_tol):
        """Tolerance of the coarse-level state solves inside the preconditioner."""
        _check(self._L.orc_set_precond_tol(self.h, pc_inner_tol), "set_precond_tol")

    def set_coarse_solve(self, mode, tol=1e-4, maxit=1000):
        """Coarsest Hessian level: 0 = dense Cholesky, 1 = plain CG to `tol`
        (Sec. 5.2).  Returns the coarse CG iterations since the last call."""
        it = C.c_long()
        _check(self._L.orc_set_coarse_solve(self.h, mode, float(tol), int(maxit), C.byref(it)),
               "set_coarse_solve")
        return it.value

    def set_yd(self, yd):
        self._yd = np.ascontiguousarray(yd, dtype=np.float64)
        _check(self._L.orc_set_yd(self.h, _p(self._yd)), "set_yd")

    def sizes(self):
        m, n = C.c_long(), C.c_long()
        Ls, Lc, ell = C.c_int(), C.c_int(), C.c_int()
        ss = np.zeros(32, dtype=np.int64)
        cs = np.zeros(32, dtype=np.int64)
        _check(self._L.orc_sizes(self.h, C.byref(m), C.byref(n), C.byref(Ls), C.byref(Lc),
                               C.byref(ell), _p(ss), _p(cs)), "sizes")
        return {"m": m.value, "n": n.value, "Ls": Ls.value, "Lc": Lc.value, "ell": ell.value,
                "state": ss[:Ls.value].tolist(), "control": cs[:Lc.value].tolist()}

    def matrix(self, which, level=0):
        """CSR of a level matrix as (rowptr, col, val, shape)."""
        wid = MATRIX[which] if isinstance(which, str) else int(which)
        r, c, z = C.c_long(), C.c_long(), C.c_long()
        _check(self._L.orc_matrix_info(self.h, wid, level, C.byref(r), C.byref(c), C.byref(z)),
               f"matrix_info {which}@{level}")
        rp = np.empty(r.value + 1, dtype=np.int32)
        ci = np.empty(z.value, dtype=np.int32)
        v = np.empty(z.value, dtype=np.float64)
        _check(self._L.orc_matrix_copy(self.h, wid, level, _p(rp), _p(ci), _p(v)), "matrix_copy")
        return rp, ci, v, (r.value, c.value)

    def scipy(self, which, level=0):
        import scipy.sparse as sp
        rp, ci, v, shape = self.matrix(which, level)
        return sp.csr_matrix((v, ci, rp), shape=shape)

    def aggregates(self, hier, level):
        rows = self.sizes()["state" if hier == 0 else "control"][level]
        agg = np.empty(rows, dtype=np.int32)
        nagg = C.c_int()
        _check(self._L.orc_aggregates(self.h, hier, level, _p(agg), C.byref(nagg)), "aggregates")
        return agg, nagg.value

    # -- operators
    def vcycle(self, level, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        _check(self._L.orc_vcycle(self.h, level, _p(b), _p(x)), "vcycle")
        return x

    def smooth(self, level, b, x0=None):
        """The level's polynomial smoother alone for A_l x = b, from x0 (None: from zero)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        _check(self._L.orc_smooth(self.h, level, _p(b), _p(x), 1 if x0 is None else 0), "smooth")
        return x

    def state_solve(self, f, level=0, tol=1e-10):
        f = np.ascontiguousarray(f, dtype=np.float64)
        y = np.zeros_like(f)
        it = C.c_long()
        _check(self._L.orc_state_solve(self.h, level, tol, _p(f), _p(y), C.byref(it)), "state_solve")
        return y, it.value

    def mass_solve(self, b, level=0):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        it = C.c_long()
        _check(self._L.orc_mass_solve(self.h, level, _p(b), _p(x), C.byref(it)), "mass_solve")
        return x, it.value

    def hessian(self, u, level=0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        hu = np.zeros_like(u)
        _check(self._L.orc_hessian(self.h, level, _p(u), _p(hu)), "hessian")
        return hu

    def precond(self, r, level=0):
        """Q_level r (Algorithm MLAS, M_u-scaled)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        _check(self._L.orc_mlas(self.h, 0, level, _p(r), _p(z)), "mlas Q")
        return z

    def R(self, r, level=0):
        """R_level r, the M_u-scaled two-grid operator T_j^-1 M_{u,j}^-1."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        _check(self._L.orc_mlas(self.h, 1, level, _p(r), _p(z)), "mlas R")
        return z

    def rhs(self):
        b = np.zeros(self.n)
        _check(self._L.orc_rhs(self.h, _p(b)), "rhs")
        return b

    def objective(self, u, grad=True):
        u = np.ascontiguousarray(u, dtype=np.float64)
        y = np.zeros(self.m)
        J = C.c_double()
        g = np.zeros(self.n) if grad else None
        _check(self._L.orc_objective(self.h, _p(u), _p(y), C.byref(J), _p(g)), "objective")
        return J.value, y, g

    def solve(self, precond=1, tol=1e-8, maxit=500):
        u = np.zeros(self.n)
        y = np.zeros(self.m)
        it, rel, happ = C.c_int(), C.c_double(), C.c_long()
        st = self._L.orc_solve(self.h, precond, tol, maxit, _p(u), _p(y), C.byref(it),
                             C.byref(rel), C.byref(happ))
        _check(st, "solve")
        return u, y, {"outer_iters": it.value, "relres": rel.value, "hessian_applies": happ.value}

    def counters(self):
        a, b, c = C.c_long(), C.c_long(), C.c_long()
        self._L.orc_counters(self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"inner_iters": a.value, "mass_iters": b.value, "hessian_applies": c.value}
