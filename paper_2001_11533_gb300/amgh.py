"""Python binding of the amgh C ABI (include/amgh.h).

Argument marshalling only: every step of the method runs in the CUDA
library libamgh.so built in this directory.  There is no fallback -- if the
library is missing, importing a function raises.  PyTorch supplies device
memory (tensors) and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamgh.so")

OK = 0
ERR = {-1: "INVALID_ARG", -2: "NOT_SETUP", -3: "CUDA", -4: "OOM", -5: "NOT_CONVERGED",
       -6: "INDEFINITE", -7: "NUMERIC", -8: "TIMEOUT"}
MATRIX = {"A": 0, "My": 1, "Myu": 2, "S": 3, "KN": 4, "Mu": 5, "P": 6, "Kfull": 7, "Mfull": 8}


class AmghError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERR.get(code, code)} ({code})")
        self.code = code


class amgh_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vertices", C.c_int64), ("coords", C.c_void_p),
                ("n_elements", C.c_int64), ("elements", C.c_void_p), ("dirichlet", C.c_void_p),
                ("on_device", C.c_int)]


class amgh_amg_opts(C.Structure):
    _fields_ = [("max_levels", C.c_int), ("hessian_levels", C.c_int), ("theta", C.c_double),
                ("coarse_max", C.c_int), ("smoother", C.c_int), ("smooth_degree", C.c_int),
                ("precision", C.c_int), ("smooth_prolongator", C.c_int), ("coarse_solve", C.c_int),
                ("fuse_coarse", C.c_int), ("autotune", C.c_int), ("aggressive", C.c_int),
                ("geometric", C.c_int), ("matrix_free", C.c_int), ("persistent_cg", C.c_int)]


class amgh_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("inner_tol", C.c_double),
                ("mass_tol", C.c_double), ("precond", C.c_int), ("ncols", C.c_int),
                ("inner_max_iter", C.c_int), ("mass_max_iter", C.c_int), ("precond_tol", C.c_double),
                ("coarse_tol", C.c_double), ("coarse_max_iter", C.c_int), ("level_fallback", C.c_int)]


class amgh_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("hessian_applies", C.c_int64),
                ("inner_iters", C.c_int64), ("mass_iters", C.c_int64), ("refinements", C.c_int64),
                ("final_relres", C.c_double), ("t_setup_s", C.c_double), ("t_solve_s", C.c_double),
                ("hessian_levels", C.c_int), ("fallbacks", C.c_int), ("coarse_iters", C.c_int64),
                ("alg_bytes", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P, _I, _I64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double
KCLASSES = 15  # AMGH_KCLASSES
_SIGS = {
    "amgh_amg_opts_default": ([_P], None),
    "amgh_solve_opts_default": ([_P], None),
    "amgh_problem_create": ([_P, _P, _D, _P, _I, _P], _I),
    "amgh_set_yd": ([_P, _P, _I], _I),
    "amgh_set_stream": ([_P, _P], _I),
    "amgh_amg_setup": ([_P, _P], _I),
    "amgh_set_solve_opts": ([_P, _P], _I),
    "amgh_hessian_apply": ([_P, _P, _P, _I], _I),
    "amgh_precond_apply": ([_P, _P, _P, _I], _I),
    "amgh_rhs": ([_P, _P], _I),
    "amgh_solve": ([_P, _P, _P, _P, _P, _P], _I),
    "amgh_solve_host": ([_P, _P, _P, _P, _P, _P], _I),
    "amgh_solve_block": ([_P, _P, _I, _P, _P, _P], _I),
    "amgh_state_solve": ([_P, _P, _P, _P], _I),
    "amgh_gradient": ([_P, _P, _P, _P], _I),
    "amgh_state_adjoint": ([_P, _P, _P], _I),
    "amgh_vcycle": ([_P, _I, _P, _P], _I),
    "amgh_state_solve_level": ([_P, _I, _P, _P, _D, _P], _I),
    "amgh_mass_solve": ([_P, _I, _P, _P, _P], _I),
    "amgh_hessian_apply_level": ([_P, _I, _P, _P], _I),
    "amgh_precond_apply_level": ([_P, _I, _I, _P, _P], _I),
    "amgh_query_sizes": ([_P, _P, _P, _P, _P, _P, _P, _P], _I),
    "amgh_get_aggregates": ([_P, _I, _I, _P, _P], _I),
    "amgh_get_matrix_info": ([_P, _I, _I, _P, _P, _P], _I),
    "amgh_get_matrix": ([_P, _I, _I, _P, _P, _P], _I),
    "amgh_get_counters": ([_P, _P], _I),
    "amgh_reset_counters": ([_P], _I),
    "amgh_get_level_counters": ([_P, _P, _P], _I),
    "amgh_kernel_timing": ([_P, _I], _I),
    "amgh_kernel_stats": ([_P, _P, _P, _P], _I),
    "amgh_kernel_class_stats": ([_P, _I, _P, _P, _P, _P], _I),
    "amgh_kernel_timing_mask": ([_P, C.c_uint], _I),
    "amgh_debug_limits": ([_I, _I, _I], _I),
    "amgh_aj_estimate": ([_P, _I, _I, _I, _P, _P], _I),
    "amgh_kuhn_apply": ([_P, _I, _P, _P], _I),
    "amgh_launch_count": ([], _I64),
    "amgh_aggregate_noalloc": ([_I, _P, _P, _P, _D, _P, _P, _P], _I),
    "amgh_dense_spd_inverse": ([_I, _P, _P, _P, _P], _I),
    "amgh_fp64_peak": ([_I, _P, _P], _I),
    "amgh_debug_grid_polls": ([_I], _I),
    "amgh_batch_create": ([_P, _I, _P], _I),
    "amgh_batch_setup": ([_P, _P], _I),
    "amgh_batch_set_workers": ([_P, _I], _I),
    "amgh_batch_set_block": ([_P, _I], _I),
    "amgh_batch_autotune": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "amgh_problem_share": ([_P, _P], _I),
    "amgh_batch_solve": ([_P, _P, _P, _P, _P, _P], _I),
    "amgh_batch_destroy": ([_P], None),
    "amgh_problem_destroy": ([_P], None),
    "amgh_status_string": ([_I], C.c_char_p),
    "amgh_last_error": ([], C.c_char_p),
}
_lib = None


def declared_symbols():
    return sorted(_SIGS)


def lib():
    """Load libamgh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the amgh path has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(code: int, what: str):
    if code != OK:
        if code in (-1, -3):  # INVALID_ARG / CUDA: say what failed (and where)
            msg = lib().amgh_last_error().decode()
            if msg:
                what = f"{what} [{msg}]"
        raise AmghError(code, what)


def _ptr(t):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def debug_limits(bulk_first_polls: int = -1, mis_round_cap: int = -1, prol_row_cap: int = -1):
    """amgh_debug_limits: lower the bounded waits' limits and the prolongator's
    register row capacity for tests (-1 = default)."""
    check(lib().amgh_debug_limits(int(bulk_first_polls), int(mis_round_cap), int(prol_row_cap)),
          "amgh_debug_limits")


def launch_count() -> int:
    return int(lib().amgh_launch_count())


def torch_empty_like(v):
    import torch
    return torch.empty_like(v, dtype=torch.float64)


def aggregate_noalloc(rowptr, col, val, theta, agg_out, stream=None):
    """amgh_aggregate_noalloc on CUDA tensors (int32 rowptr/col, float64 val);
    writes agg_out (int32, n) and returns the number of aggregates."""
    n = int(rowptr.numel()) - 1
    nagg = C.c_int32()
    check(lib().amgh_aggregate_noalloc(n, _ptr(rowptr), _ptr(col), _ptr(val), float(theta),
                                       C.c_void_p(stream) if stream else None, _ptr(agg_out),
                                       C.byref(nagg)), "amgh_aggregate_noalloc")
    return nagg.value


ERR_INDEFINITE = -6
ERR_TIMEOUT = -8


def dense_spd_inverse(a, inv_out, stream=None):
    """amgh_dense_spd_inverse on CUDA float64 tensors (n x n, row-major; the
    lower triangle of a is read).  Returns (status, info): status 0 or
    ERR_INDEFINITE (-6), info the 1-based row of the first non-positive pivot;
    other errors raise AmghError."""
    n = int(a.shape[0])
    info = C.c_int32()
    st = lib().amgh_dense_spd_inverse(n, _ptr(a), _ptr(inv_out), C.c_void_p(stream) if stream else None,
                                      C.byref(info))
    if st not in (0, ERR_INDEFINITE):
        check(st, "amgh_dense_spd_inverse")
    return st, info.value


def debug_grid_polls(polls: int = -1):
    """amgh_debug_grid_polls: poll limit of every software grid barrier wait
    (-1 = default); a test hook for the timeout path."""
    check(lib().amgh_debug_grid_polls(int(polls)), "amgh_debug_grid_polls")


def fp64_peak(kind: int, stream=None) -> float:
    """amgh_fp64_peak: measured FP64 TFLOP/s, kind 0 = FMA pipe, 1 = mma.m8n8k4.f64."""
    t = C.c_double()
    check(lib().amgh_fp64_peak(int(kind), C.c_void_p(stream) if stream else None, C.byref(t)), "amgh_fp64_peak")
    return t.value


def _fill(o, kw):
    names = {k for k, _ in o._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"{type(o).__name__} has no field {k!r}")
        setattr(o, k, v)
    return o


def amg_opts(**kw) -> amgh_amg_opts:
    o = amgh_amg_opts()
    lib().amgh_amg_opts_default(C.byref(o))
    return _fill(o, kw)


def solve_opts(**kw) -> amgh_solve_opts:
    o = amgh_solve_opts()
    lib().amgh_solve_opts_default(C.byref(o))
    return _fill(o, kw)


class Problem:
    """One control problem resident on the current CUDA device.

    Construct from host numpy arrays (`on_device=False`) or CUDA tensors
    (`on_device=True`); see include/amgh.h for layouts.
    """

    def __init__(self, dim, coords, elements, dirichlet, kappa, beta, y_d, on_device=None,
                 stream=None):
        import torch
        L = lib()
        if on_device is None:
            on_device = not isinstance(coords, np.ndarray)
        self._keep = (coords, elements, dirichlet, kappa, y_d)
        mesh = amgh_mesh(dim, int(coords.shape[0]), _ptr(coords), int(elements.shape[0]),
                         _ptr(elements), _ptr(dirichlet), 1 if on_device else 0)
        h = C.c_void_p()
        self.h = None
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        check(L.amgh_problem_create(C.byref(mesh), _ptr(kappa), float(beta), _ptr(y_d),
                                    1 if on_device else 0, C.byref(h)), "amgh_problem_create")
        self.h = h
        if stream is not None:
            check(L.amgh_set_stream(self.h, C.c_void_p(stream)), "amgh_set_stream")
        self._keep = None
        self.beta = float(beta)
        self.dim = dim

    @classmethod
    def from_workload(cls, w, device=True, y_index=0):
        """Upload a workloads.Workload (as CUDA tensors when device=True)."""
        yd = w.y_d if w.y_d.ndim == 1 else w.y_d[y_index]
        arrs = [np.ascontiguousarray(w.coords, dtype=np.float64),
                np.ascontiguousarray(w.elements, dtype=np.int32),
                np.ascontiguousarray(w.dirichlet, dtype=np.uint8),
                np.ascontiguousarray(w.kappa, dtype=np.float64),
                np.ascontiguousarray(yd, dtype=np.float64)]
        if device:
            import torch
            arrs = [torch.from_numpy(a).cuda() for a in arrs]
            torch.cuda.synchronize()
        return cls(w.dim, arrs[0], arrs[1], arrs[2], arrs[3], w.beta, arrs[4], on_device=device)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "h", None):
            lib().amgh_problem_destroy(self.h)
            self.h = None

    # -- setup and options
    def share(self, stream=None):
        """A second handle on this problem's matrices and hierarchies with its
        own work space (amgh_problem_share); keeps this problem alive."""
        h = C.c_void_p()
        check(lib().amgh_problem_share(self.h, C.byref(h)), "amgh_problem_share")
        q = Problem.__new__(Problem)
        q.h, q.beta, q.dim, q.sizes, q._parent = h, self.beta, self.dim, dict(self.sizes), self
        if stream is not None:
            q.set_stream(stream)
        return q

    def amg_setup(self, **kw):
        o = amg_opts(**kw)
        check(lib().amgh_amg_setup(self.h, C.byref(o)), "amgh_amg_setup")
        self.sizes = self.query_sizes()
        return self

    def set_solve_opts(self, **kw):
        o = solve_opts(**kw)
        check(lib().amgh_set_solve_opts(self.h, C.byref(o)), "amgh_set_solve_opts")

    def set_stream(self, stream):
        check(lib().amgh_set_stream(self.h, C.c_void_p(stream)), "amgh_set_stream")

    def set_yd(self, y_d):
        on_dev = not isinstance(y_d, np.ndarray)
        check(lib().amgh_set_yd(self.h, _ptr(y_d), 1 if on_dev else 0), "amgh_set_yd")

    def query_sizes(self):
        m, n = C.c_int64(), C.c_int64()
        Ls, Lc, ell = C.c_int(), C.c_int(), C.c_int()
        ss = np.zeros(32, dtype=np.int64)
        cs = np.zeros(32, dtype=np.int64)
        check(lib().amgh_query_sizes(self.h, C.byref(m), C.byref(n), C.byref(Ls), C.byref(Lc),
                                     C.byref(ell), _ptr(ss), _ptr(cs)), "amgh_query_sizes")
        return {"m": m.value, "n": n.value, "Ls": Ls.value, "Lc": Lc.value, "ell": ell.value,
                "state": ss[:Ls.value].tolist(), "control": cs[:Lc.value].tolist()}

    # -- helpers
    def _new(self, k, like=None):
        import torch
        return torch.empty(k, dtype=torch.float64, device="cuda")

    # -- the hot path
    @staticmethod
    def _cols(v):
        """(n,) or (k, n) contiguous tensor: k stacked vectors, column-major n x k."""
        if not v.is_contiguous():
            raise ValueError("vectors must be contiguous (k, n) or (n,) tensors")
        return 1 if v.dim() == 1 else int(v.shape[0])

    def hessian_apply(self, u, out=None):
        """H u for u of shape (n,) or (k, n); k > 1 runs the block solver."""
        out = torch_empty_like(u) if out is None else out
        check(lib().amgh_hessian_apply(self.h, _ptr(u), _ptr(out), self._cols(u)), "amgh_hessian_apply")
        return out

    def precond_apply(self, r, out=None):
        """Q_0 r for r of shape (n,) or (k, n); k > 1 runs the block solver."""
        out = torch_empty_like(r) if out is None else out
        check(lib().amgh_precond_apply(self.h, _ptr(r), _ptr(out), self._cols(r)), "amgh_precond_apply")
        return out

    def rhs(self):
        b = self._new(self.sizes["n"])
        check(lib().amgh_rhs(self.h, _ptr(b)), "amgh_rhs")
        return b

    def solve(self, u0=None, want_y=True, raise_on_error=True, **kw):
        o = solve_opts(**kw)
        u = self._new(self.sizes["n"])
        y = self._new(self.sizes["m"]) if want_y else None
        info = amgh_solve_info()
        st = lib().amgh_solve(self.h, _ptr(u0), _ptr(u), _ptr(y), C.byref(o), C.byref(info))
        if raise_on_error:
            check(st, "amgh_solve")
        return u, y, info.as_dict()

    def solve_block(self, yds, raise_on_error=True, **kw):
        """Controls for k desired states yds (CUDA float64, shape (k, n_vertices))
        solved together by the block solver; returns ((k, n) controls, info, status)."""
        import torch
        yds = yds.contiguous()
        k = int(yds.shape[0])
        u = torch.empty((k, self.sizes["n"]), dtype=torch.float64, device=yds.device)
        info = amgh_solve_info()
        o = solve_opts(**kw)
        st = lib().amgh_solve_block(self.h, _ptr(yds), k, _ptr(u), C.byref(o), C.byref(info))
        if raise_on_error:
            check(st, "amgh_solve_block")
        return u, info.as_dict(), st

    def solve_host(self, u0=None, want_y=True, **kw):
        o = solve_opts(**kw)
        u = np.zeros(self.sizes["n"])
        y = np.zeros(self.sizes["m"]) if want_y else None
        info = amgh_solve_info()
        check(lib().amgh_solve_host(self.h, _ptr(u0), _ptr(u), _ptr(y), C.byref(o), C.byref(info)),
              "amgh_solve_host")
        return u, y, info.as_dict()

    def state_solve(self, u):
        y = self._new(self.sizes["m"])
        J = C.c_double()
        check(lib().amgh_state_solve(self.h, _ptr(u), _ptr(y), C.byref(J)), "amgh_state_solve")
        return y, J.value

    def gradient(self, u, y):
        g = self._new(self.sizes["n"])
        check(lib().amgh_gradient(self.h, _ptr(u), _ptr(y), _ptr(g)), "amgh_gradient")
        return g

    def state_adjoint(self, w):
        g = self._new(self.sizes["n"])
        check(lib().amgh_state_adjoint(self.h, _ptr(w), _ptr(g)), "amgh_state_adjoint")
        return g

    def state_only(self, u):
        """y = A^-1 M_yu u without evaluating J."""
        y = self._new(self.sizes["m"])
        check(lib().amgh_state_solve(self.h, _ptr(u), _ptr(y), None), "amgh_state_solve")
        return y

    # -- level-wise pieces
    def vcycle(self, level, b):
        x = self._new(b.numel())
        check(lib().amgh_vcycle(self.h, level, _ptr(b), _ptr(x)), "amgh_vcycle")
        return x

    def state_solve_level(self, level, f, tol):
        y = self._new(f.numel())
        it = C.c_int64()
        check(lib().amgh_state_solve_level(self.h, level, _ptr(f), _ptr(y), float(tol), C.byref(it)),
              "amgh_state_solve_level")
        return y, it.value

    def mass_solve(self, level, b):
        x = self._new(b.numel())
        it = C.c_int64()
        check(lib().amgh_mass_solve(self.h, level, _ptr(b), _ptr(x), C.byref(it)), "amgh_mass_solve")
        return x, it.value

    def hessian_apply_level(self, level, v):
        hv = self._new(v.numel())
        check(lib().amgh_hessian_apply_level(self.h, level, _ptr(v), _ptr(hv)),
              "amgh_hessian_apply_level")
        return hv

    def precond_apply_level(self, which, level, b):
        z = self._new(b.numel())
        check(lib().amgh_precond_apply_level(self.h, which, level, _ptr(b), _ptr(z)),
              "amgh_precond_apply_level")
        return z

    # -- inspection
    def aggregates(self, hier, level):
        rows = self.sizes["state" if hier == 0 else "control"][level]
        agg = np.empty(rows, dtype=np.int32)
        nagg = C.c_int32()
        check(lib().amgh_get_aggregates(self.h, hier, level, _ptr(agg), C.byref(nagg)),
              "amgh_get_aggregates")
        return agg, nagg.value

    def matrix(self, which, level=0):
        wid = MATRIX[which] if isinstance(which, str) else int(which)
        r, c, z = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().amgh_get_matrix_info(self.h, wid, level, C.byref(r), C.byref(c), C.byref(z)),
              "amgh_get_matrix_info")
        rp = np.empty(r.value + 1, dtype=np.int32)
        ci = np.empty(z.value, dtype=np.int32)
        v = np.empty(z.value, dtype=np.float64)
        check(lib().amgh_get_matrix(self.h, wid, level, _ptr(rp), _ptr(ci), _ptr(v)), "amgh_get_matrix")
        return rp, ci, v, (r.value, c.value)

    def counters(self):
        info = amgh_solve_info()
        check(lib().amgh_get_counters(self.h, C.byref(info)), "amgh_get_counters")
        return info.as_dict()

    def level_counters(self):
        a = np.zeros(32, dtype=np.int64)
        b = np.zeros(32, dtype=np.int64)
        check(lib().amgh_get_level_counters(self.h, _ptr(a), _ptr(b)), "amgh_get_level_counters")
        return {"inner": a[:self.sizes["Ls"]].tolist(), "mass": b[:self.sizes["Lc"]].tolist()}

    def reset_counters(self):
        check(lib().amgh_reset_counters(self.h), "amgh_reset_counters")

    def kernel_timing(self, enable=True):
        check(lib().amgh_kernel_timing(self.h, 1 if enable else 0), "amgh_kernel_timing")

    def kernel_stats(self):
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        check(lib().amgh_kernel_stats(self.h, C.byref(n), C.byref(ms), C.byref(b)), "amgh_kernel_stats")
        return {"launches": n.value, "ms": ms.value, "bytes": b.value}

    def aj_estimate(self, level, v0, weighted=False, iters=30):
        """a~_j (weighted False) or a_j (True) on `level` by the power method
        from the CUDA vector v0 (amgh_aj_estimate)."""
        est = C.c_double()
        check(lib().amgh_aj_estimate(self.h, int(level), 1 if weighted else 0, int(iters), _ptr(v0),
                                     C.byref(est)), "amgh_aj_estimate")
        return est.value

    def kuhn_apply(self, x, out=None):
        """A x by the matrix-free Kuhn-cube operator (amgh_kuhn_apply); x float64
        or float32 CUDA tensor of the m states."""
        import torch
        out = torch.empty_like(x) if out is None else out
        prec32 = 1 if x.dtype == torch.float32 else 0
        check(lib().amgh_kuhn_apply(self.h, prec32, _ptr(x), _ptr(out)), "amgh_kuhn_apply")
        return out

    def kernel_timing_mask(self, mask):
        """Time only the kernel classes whose bit is set (amgh_kernel_timing_mask)."""
        check(lib().amgh_kernel_timing_mask(self.h, C.c_uint(mask)), "amgh_kernel_timing_mask")

    def kernel_class_stats(self):
        """{class name: {launches, ms, bytes}} for every kernel class (amgh_kernel_class_stats)."""
        out = {}
        for c in range(KCLASSES):
            n, ms, b, name = C.c_int64(), C.c_double(), C.c_double(), C.c_char_p()
            check(lib().amgh_kernel_class_stats(self.h, c, C.byref(n), C.byref(ms), C.byref(b), C.byref(name)),
                  "amgh_kernel_class_stats")
            out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": b.value}
        return out


class Batch:
    """Many independent problems, several desired states each, solved
    concurrently (amgh_batch_*): per problem up to `workers` slots (0 = one per
    desired state, or one per problem with block=True), each with its own CUDA
    stream and native host thread; block=True solves a slot's desired states
    together with the block solver."""

    def __init__(self, problems, workers=0, block=False):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = C.c_void_p()
        check(lib().amgh_batch_create(arr, len(self.problems), C.byref(h)), "amgh_batch_create")
        self.h = h
        check(lib().amgh_batch_set_workers(self.h, int(workers)), "amgh_batch_set_workers")
        check(lib().amgh_batch_set_block(self.h, 1 if block else 0), "amgh_batch_set_block")

    def set_block(self, block=True):
        check(lib().amgh_batch_set_block(self.h, 1 if block else 0), "amgh_batch_set_block")
        return self

    def set_workers(self, workers):
        check(lib().amgh_batch_set_workers(self.h, int(workers)), "amgh_batch_set_workers")
        return self

    CANDIDATES = ("columns", "block K=8", "block K=4 x 2 slots", "block K=2 x 4 slots")

    def autotune(self, yds, **kw):
        """amgh_batch_autotune: time the four slot / block-width candidates on
        these desired states and keep the fastest; returns (choice, seconds)."""
        import torch
        np_ = len(self.problems)
        yds = [y.contiguous() for y in yds]
        us = [torch.empty_like(y) for y in yds]
        ycols = (C.c_int * np_)(*[int(y.shape[0]) for y in yds])
        yptr = (C.c_void_p * np_)(*[y.data_ptr() for y in yds])
        uptr = (C.c_void_p * np_)(*[u.data_ptr() for u in us])
        times = (C.c_double * 4)()
        choice = C.c_int()
        o = solve_opts(**kw)
        torch.cuda.synchronize()
        check(lib().amgh_batch_autotune(self.h, yptr, ycols, uptr, C.byref(o), times, C.byref(choice)),
              "amgh_batch_autotune")
        return self.CANDIDATES[choice.value], dict(zip(self.CANDIDATES, list(times)))

    def setup(self, **kw):
        o = amg_opts(**kw)
        check(lib().amgh_batch_setup(self.h, C.byref(o)), "amgh_batch_setup")
        for p in self.problems:
            p.sizes = p.query_sizes()
        return self

    def solve(self, yds, raise_on_error=True, **kw):
        """yds[p]: CUDA float64 tensor (ncols, n_vertices) of desired states;
        returns a list of (ncols, n) controls and the per-problem counters."""
        import torch
        np_ = len(self.problems)
        yds = [y.contiguous() for y in yds]
        us = [torch.empty_like(y) for y in yds]
        ycols = (C.c_int * np_)(*[int(y.shape[0]) for y in yds])
        yptr = (C.c_void_p * np_)(*[y.data_ptr() for y in yds])
        uptr = (C.c_void_p * np_)(*[u.data_ptr() for u in us])
        infos = (amgh_solve_info * np_)()
        o = solve_opts(**kw)
        # the batch runs on its own streams: inputs and outputs must be ready
        torch.cuda.current_stream().synchronize()
        st = lib().amgh_batch_solve(self.h, yptr, ycols, uptr, C.byref(o), infos)
        if raise_on_error:
            check(st, "amgh_batch_solve")
        return us, [i.as_dict() for i in infos], st

    def close(self):
        if getattr(self, "h", None):
            lib().amgh_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
