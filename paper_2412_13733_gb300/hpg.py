"""Thin ctypes binding of libhpg (include/hpg.h): same names, argument marshalling only.

Every step of the solve runs in libhpg's CUDA kernels; this module only
converts numpy arrays and Python callables to the C ABI.  It raises if the
compiled library is missing -- there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhpg.so")

HPG_OBSTACLE_UPPER, HPG_OBSTACLE_LOWER, HPG_GRADIENT = 0, 1, 2
HPG_FP64, HPG_MIXED = 0, 1
HPG_SCHUR, HPG_FGMRES_PD, HPG_FGMRES_PLPD, HPG_FGMRES_PF = 0, 1, 2, 3
HPG_MAX_ALPHA = 128
KERNEL_CLASSES = ["eval", "residual", "factor", "precond", "bapply", "fdm", "schur", "ortho", "newton_apply",
                  "update"]
STATUS = ["HPG_OK", "HPG_ERR_ARG", "HPG_ERR_OOM", "HPG_ERR_CUDA", "HPG_ERR_NEWTON_CAP", "HPG_ERR_KRYLOV_CAP",
          "HPG_ERR_NONFINITE", "HPG_ERR_NOT_SPD", "HPG_ERR_TIMEOUT", "HPG_ERR_INFEASIBLE_BC", "HPG_ERR_STATE",
          "HPG_ERR_BUSY"]


class hpg_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("newton_tol", C.c_double), ("newton_max", C.c_int),
                ("krylov_max", C.c_int), ("krylov_rtol", C.c_double), ("precision", C.c_int),
                ("ls_max", C.c_int), ("refine_max", C.c_int), ("timing", C.c_int), ("graphs", C.c_int),
                ("fdm_tile_f32", C.c_int), ("fdm_tile_f64", C.c_int), ("strategy", C.c_int),
                ("inner_max", C.c_int), ("krylov_f32", C.c_int), ("ainv_pcg", C.c_int), ("ainv_rtol", C.c_double),
                ("fdm_tune_batch", C.c_int)]


class hpg_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("alpha_steps", C.c_int), ("newton_total", C.c_int),
                ("newton_per_step", C.c_int * HPG_MAX_ALPHA), ("krylov_total", C.c_longlong),
                ("refine_total", C.c_int), ("ls_fail", C.c_int), ("krylov_cap_hits", C.c_int),
                ("final_residual", C.c_double), ("solve_ms", C.c_double), ("n_u", C.c_longlong),
                ("n_psi", C.c_longlong), ("kernel_launches", C.c_longlong), ("h2d_bytes", C.c_longlong),
                ("fdm_tile_f32", C.c_int), ("fdm_tile_f64", C.c_int), ("fgmres_total", C.c_longlong),
                ("ainv_total", C.c_longlong), ("ainv_iters", C.c_longlong), ("fp64_from_step", C.c_int),
                ("fp64_newton_steps", C.c_int)]


HPG_QVI_MAX_FP = 64


class hpg_qvi_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("g0", C.c_double), ("tol", C.c_double), ("t_tol", C.c_double),
                ("max_fp", C.c_int), ("nq", C.c_int), ("t_newton_max", C.c_int), ("t_krylov_max", C.c_int),
                ("t_krylov_rtol", C.c_double)]


class hpg_qvi_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("converged", C.c_int), ("newton_total", C.c_int),
                ("t_newton_total", C.c_int), ("t_krylov_total", C.c_longlong),
                ("du_h1", C.c_double * HPG_QVI_MAX_FP), ("newton_per_fp", C.c_int * HPG_QVI_MAX_FP),
                ("t_newton_per_fp", C.c_int * HPG_QVI_MAX_FP), ("t_residual", C.c_double),
                ("solve_ms", C.c_double), ("kernel_launches", C.c_longlong), ("krylov_total", C.c_longlong)]


FIELD_FN = C.CFUNCTYPE(None, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)

_P = C.POINTER
_d = C.c_double
_pd = _P(C.c_double)
_sz = C.c_size_t
_ctx = C.c_void_p

SIGNATURES = {
    "hpg_create": ([_P(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "hpg_destroy": ([_ctx], C.c_int),
    "hpg_status_str": ([C.c_int], C.c_char_p),
    "hpg_last_error": ([_ctx], C.c_char_p),
    "hpg_default_params": ([_P(hpg_params)], None),
    "hpg_problem_create": ([_ctx, C.c_int, _pd, _pd, _P(C.c_int), C.c_int, C.c_int, _P(C.c_int)], C.c_int),
    "hpg_problem_free": ([_ctx, C.c_int], C.c_int),
    "hpg_problem_sizes": ([_ctx, C.c_int, _P(_sz), _P(_sz), _P(_sz), _P(_sz)], C.c_int),
    "hpg_set_rhs": ([_ctx, C.c_int, FIELD_FN, C.c_void_p], C.c_int),
    "hpg_set_rhs_const": ([_ctx, C.c_int, _d], C.c_int),
    "hpg_set_constraint": ([_ctx, C.c_int, FIELD_FN, C.c_void_p], C.c_int),
    "hpg_quad_points": ([_ctx, C.c_int, _pd, _sz], C.c_int),
    "hpg_set_constraint_values": ([_ctx, C.c_int, _pd, _sz], C.c_int),
    "hpg_set_dirichlet": ([_ctx, C.c_int, FIELD_FN, C.c_void_p], C.c_int),
    "hpg_set_alpha_schedule": ([_ctx, C.c_int, _d, _d], C.c_int),
    "hpg_set_alpha_list": ([_ctx, C.c_int, _pd, C.c_int], C.c_int),
    "hpg_set_alpha_growth": ([_ctx, C.c_int, _d, _d, _d, C.c_int, C.c_int], C.c_int),
    "hpg_set_params": ([_ctx, C.c_int, _P(hpg_params)], C.c_int),
    "hpg_solve": ([_ctx, C.c_int], C.c_int),
    "hpg_solve_batch": ([_ctx, _P(C.c_int), C.c_int], C.c_int),
    "hpg_set_concurrency": ([_ctx, C.c_int], C.c_int),
    "hpg_get_u": ([_ctx, C.c_int, _pd, _sz], C.c_int),
    "hpg_get_psi": ([_ctx, C.c_int, _pd, _sz], C.c_int),
    "hpg_get_stats": ([_ctx, C.c_int, _P(hpg_stats)], C.c_int),
    "hpg_eval_u": ([_ctx, C.c_int, _pd, C.c_int, _pd], C.c_int),
    "hpg_feasible_u": ([_ctx, C.c_int, _pd, _sz], C.c_int),
    "hpg_get_kernel_times": ([_ctx, C.c_int, _pd, _P(C.c_longlong), C.c_int], C.c_int),
    "hpg_reset_kernel_times": ([_ctx, C.c_int], C.c_int),
    "hpg_set_state": ([_ctx, C.c_int, _pd, _pd, _pd, _d], C.c_int),
    "hpg_residual": ([_ctx, C.c_int, _pd, _sz, _pd], C.c_int),
    "hpg_apply_newton": ([_ctx, C.c_int, _pd, _pd, _sz], C.c_int),
    "hpg_apply_stiffness_inv": ([_ctx, C.c_int, C.c_int, _pd, _pd, _sz], C.c_int),
    "hpg_factor_precond": ([_ctx, C.c_int, C.c_int, _pd, _sz], C.c_int),
    "hpg_apply_precond_inv": ([_ctx, C.c_int, C.c_int, _pd, _pd, _sz], C.c_int),
    "hpg_apply_schur": ([_ctx, C.c_int, C.c_int, _pd, _pd, _sz], C.c_int),
    "hpg_newton_direction": ([_ctx, C.c_int, C.c_int, _d, _pd, _sz, _P(C.c_int)], C.c_int),
    "hpg_launch_kernel": ([_ctx, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    "hpg_fdm_tile_count": ([C.c_int], C.c_int),
    "hpg_stiffness_solve_pcg": ([_ctx, C.c_int, C.c_int, _d, _pd, _pd, _sz, _d, _d, C.c_int, _P(C.c_int)], C.c_int),
    "hpg_launch_kernel_batch": ([_ctx, _P(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    "hpg_apply_stiffness_inv_noalloc": ([_ctx, C.c_int, _d, C.c_void_p, C.c_void_p, _sz], C.c_int),
    "hpg_server_start": ([_ctx, C.c_int, _sz], C.c_int),
    "hpg_server_stop": ([_ctx], C.c_int),
    "hpg_submit": ([_ctx, C.c_int, _P(C.c_longlong)], C.c_int),
    "hpg_poll": ([_ctx, C.c_longlong, _P(C.c_int), _P(C.c_int)], C.c_int),
    "hpg_wait": ([_ctx, C.c_longlong, _d, _P(C.c_int)], C.c_int),
    "hpg_ticket_times": ([_ctx, C.c_longlong, _pd], C.c_int),
    "hpg_server_memory": ([_ctx, C.c_int, _P(_sz), _P(_sz)], C.c_int),
    "hpg_ticket_error": ([_ctx, C.c_longlong, C.c_char_p, _sz], C.c_int),
    "hpg_server_policy": ([_ctx, C.c_int], C.c_int),
    "hpg_l2_error": ([_ctx, C.c_int, _pd, _sz, _pd, _pd], C.c_int),
    "hpg_measure_fma_peak": ([_ctx, C.c_int, _pd, _P(C.c_int)], C.c_int),
    "hpg_qvi_default_params": ([_P(hpg_qvi_params)], C.c_int),
    "hpg_qvi_points": ([_ctx, C.c_int, C.c_int, _pd, _sz], C.c_int),
    "hpg_qvi_solve": ([_ctx, C.c_int, _P(hpg_qvi_params), _pd, _pd, _sz, _pd, _pd, _sz, _P(hpg_qvi_stats)],
                      C.c_int),
    "hpg_qvi_get_T": ([_ctx, C.c_int, _pd, _sz], C.c_int),
}

_lib = None


def lib():
    """Load libhpg.so (built in-tree by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhpg.so not built ({LIB_PATH}); run python -m paper_2412_13733_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class HpgError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{STATUS[code] if 0 <= code < len(STATUS) else code}: {msg}")


def _dptr(a):
    return a.ctypes.data_as(_pd)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def field(fn):
    """Wrap a Python field f(X: (npts, dim) array) -> (npts,) as an hpg_field_fn."""
    def cb(npts, dim, x, out, user):
        X = np.ctypeslib.as_array(x, shape=(npts * dim,)).reshape(npts, dim)
        np.ctypeslib.as_array(out, shape=(npts,))[:] = np.asarray(fn(X.copy()), dtype=np.float64)
    return FIELD_FN(cb)


class Context:
    """hpg_ctx on one CUDA device (stream: optional cudaStream_t handle as int)."""

    def __init__(self, device=0, stream=None):
        self.L = lib()
        h = C.c_void_p()
        rc = self.L.hpg_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None)
        if rc != 0:
            raise HpgError(rc, "hpg_create")
        self.h = h
        self._keep = []

    def check(self, rc, what=""):
        if rc != 0:
            raise HpgError(rc, f"{what}: {self.L.hpg_last_error(self.h).decode()}")
        return rc

    def solve_batch(self, problems, check=True):
        ids = (C.c_int * len(problems))(*[p.pid for p in problems])
        rc = self.L.hpg_solve_batch(self.h, ids, len(problems))
        if check:
            self.check(rc, "hpg_solve_batch")
        return rc

    # request loop
    def server_start(self, workers=8, budget_bytes=0):
        self.check(self.L.hpg_server_start(self.h, int(workers), int(budget_bytes)), "hpg_server_start")

    def server_stop(self):
        self.check(self.L.hpg_server_stop(self.h), "hpg_server_stop")

    def submit(self, problem):
        t = C.c_longlong()
        self.check(self.L.hpg_submit(self.h, problem.pid, C.byref(t)), "hpg_submit")
        return t.value

    def poll(self, ticket):
        done, res = C.c_int(), C.c_int()
        self.check(self.L.hpg_poll(self.h, C.c_longlong(ticket), C.byref(done), C.byref(res)), "hpg_poll")
        return bool(done.value), res.value

    def wait(self, ticket, timeout_ms=60000.0):
        res = C.c_int()
        rc = self.L.hpg_wait(self.h, C.c_longlong(ticket), float(timeout_ms), C.byref(res))
        if rc != 0:
            raise HpgError(rc, "hpg_wait")
        return res.value

    def ticket_times(self, ticket):
        t = (C.c_double * 3)()
        self.check(self.L.hpg_ticket_times(self.h, C.c_longlong(ticket), t), "hpg_ticket_times")
        return tuple(t)

    def server_policy(self, policy):
        self.check(self.L.hpg_server_policy(self.h, int(policy)), "hpg_server_policy")

    def ticket_error(self, ticket):
        buf = C.create_string_buffer(512)
        self.check(self.L.hpg_ticket_error(self.h, C.c_longlong(ticket), buf, 512), "hpg_ticket_error")
        return buf.value.decode()

    def server_memory(self, problem=None):
        a, b = _sz(), _sz()
        self.check(self.L.hpg_server_memory(self.h, problem.pid if problem else 0, C.byref(a),
                                            C.byref(b) if problem else None))
        return a.value, (b.value if problem else None)

    def launch_kernel_batch(self, problems, name, precision=HPG_FP64, reps=1):
        """Replay `reps` launches of one kernel class over a lockstep group of solved problems."""
        cls = KERNEL_CLASSES.index(name) if isinstance(name, str) else int(name)
        ids = (C.c_int * len(problems))(*[p.pid for p in problems])
        self.check(self.L.hpg_launch_kernel_batch(self.h, ids, len(problems), cls, int(precision), int(reps)),
                   "hpg_launch_kernel_batch")

    def fma_peak(self, precision):
        """Measured SIMT FMA throughput (TFLOP/s) and SM count of the device."""
        t, n = C.c_double(), C.c_int()
        self.check(self.L.hpg_measure_fma_peak(self.h, int(precision), C.byref(t), C.byref(n)),
                   "hpg_measure_fma_peak")
        return t.value, n.value

    def set_concurrency(self, n):
        self.check(self.L.hpg_set_concurrency(self.h, int(n)), "hpg_set_concurrency")

    def close(self):
        if self.h:
            self.L.hpg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fdm_tile_count(precision):
    """Number of fast-diagonalisation pass variants (valid hpg_params.fdm_tile_f32/_f64)."""
    return int(lib().hpg_fdm_tile_count(int(precision)))


def default_params(**kw):
    p = hpg_params()
    lib().hpg_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Problem:
    """One hpG problem in a Context (argument marshalling over the C ABI)."""

    def __init__(self, ctx, dim, lo, hi, cells, p, kind):
        self.pid = None
        self.ctx, self.L = ctx, ctx.L
        pid = C.c_int()
        lo = _f64(lo)
        hi = _f64(hi)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        ctx.check(self.L.hpg_problem_create(ctx.h, int(dim), _dptr(lo), _dptr(hi),
                                            cells.ctypes.data_as(_P(C.c_int)), int(p), int(kind), C.byref(pid)),
                  "hpg_problem_create")
        self.pid = pid.value
        self.dim = dim
        self._p = int(p)
        self.cells = int(np.prod(cells))
        a, b, c, d = (_sz() for _ in range(4))
        ctx.check(self.L.hpg_problem_sizes(ctx.h, self.pid, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        self.n_u_full, self.n_u, self.n_psi, self.n_quad = a.value, b.value, c.value, d.value
        self._cbs = []

    # data
    def set_rhs(self, f):
        if callable(f):
            cb = field(f)
            self._cbs.append(cb)
            self.ctx.check(self.L.hpg_set_rhs(self.ctx.h, self.pid, cb, None), "hpg_set_rhs")
        else:
            self.ctx.check(self.L.hpg_set_rhs_const(self.ctx.h, self.pid, float(f)), "hpg_set_rhs_const")

    def quad_points(self):
        out = np.zeros(self.n_quad * self.dim)
        self.ctx.check(self.L.hpg_quad_points(self.ctx.h, self.pid, _dptr(out), out.size), "hpg_quad_points")
        return out.reshape(self.n_quad, self.dim)

    def set_constraint(self, phi):
        cb = field(phi)
        self._cbs.append(cb)
        self.ctx.check(self.L.hpg_set_constraint(self.ctx.h, self.pid, cb, None), "hpg_set_constraint")

    def set_constraint_values(self, vals):
        v = _f64(vals)
        self.ctx.check(self.L.hpg_set_constraint_values(self.ctx.h, self.pid, _dptr(v), v.size),
                       "hpg_set_constraint_values")

    def set_dirichlet(self, g):
        cb = field(g) if g is not None else FIELD_FN()
        if g is not None:
            self._cbs.append(cb)
        self.ctx.check(self.L.hpg_set_dirichlet(self.ctx.h, self.pid, cb, None), "hpg_set_dirichlet")

    def set_alphas(self, alphas):
        a = _f64(alphas)
        self.ctx.check(self.L.hpg_set_alpha_list(self.ctx.h, self.pid, _dptr(a), a.size), "hpg_set_alpha_list")

    def set_alpha_growth(self, a1, growth, cap, max_steps=HPG_MAX_ALPHA, cap_twice=False):
        self.ctx.check(self.L.hpg_set_alpha_growth(self.ctx.h, self.pid, float(a1), float(growth), float(cap),
                                                   int(max_steps), int(bool(cap_twice))), "hpg_set_alpha_growth")

    def set_alpha_schedule(self, a1, cap):
        self.ctx.check(self.L.hpg_set_alpha_schedule(self.ctx.h, self.pid, float(a1), float(cap)))

    def set_params(self, params):
        self.ctx.check(self.L.hpg_set_params(self.ctx.h, self.pid, C.byref(params)), "hpg_set_params")

    # solve
    def solve(self, check=True):
        rc = self.L.hpg_solve(self.ctx.h, self.pid)
        if check:
            self.ctx.check(rc, "hpg_solve")
        return rc

    def u(self):
        out = np.zeros(self.n_u_full)
        self.ctx.check(self.L.hpg_get_u(self.ctx.h, self.pid, _dptr(out), out.size), "hpg_get_u")
        return out

    def psi(self):
        out = np.zeros(self.n_psi)
        self.ctx.check(self.L.hpg_get_psi(self.ctx.h, self.pid, _dptr(out), out.size), "hpg_get_psi")
        return out

    def stats(self):
        s = hpg_stats()
        self.ctx.check(self.L.hpg_get_stats(self.ctx.h, self.pid, C.byref(s)))
        d = {k: getattr(s, k) for k, _ in hpg_stats._fields_ if k != "newton_per_step"}
        d["newton_per_step"] = list(s.newton_per_step[:s.alpha_steps])
        return d

    def eval_u(self, X):
        X = _f64(X)
        out = np.zeros(X.shape[0])
        self.ctx.check(self.L.hpg_eval_u(self.ctx.h, self.pid, _dptr(X), X.shape[0], _dptr(out)), "hpg_eval_u")
        return out

    def l2_error(self, u_ref):
        """(||u_h - u_ref||_L2, ||u_ref||_L2) of the last solve, u_ref full coefficients."""
        r = _f64(u_ref)
        e, n = C.c_double(), C.c_double()
        self.ctx.check(self.L.hpg_l2_error(self.ctx.h, self.pid, _dptr(r), r.size, C.byref(e), C.byref(n)),
                       "hpg_l2_error")
        return e.value, n.value

    def feasible_u(self):
        out = np.zeros(self.n_quad)
        self.ctx.check(self.L.hpg_feasible_u(self.ctx.h, self.pid, _dptr(out), out.size), "hpg_feasible_u")
        return out

    def kernel_times(self):
        ms = np.zeros(len(KERNEL_CLASSES))
        ln = (C.c_longlong * len(KERNEL_CLASSES))()
        self.ctx.check(self.L.hpg_get_kernel_times(self.ctx.h, self.pid, _dptr(ms), ln, len(KERNEL_CLASSES)))
        return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def launch_kernel(self, name, precision=HPG_FP64, reps=1):
        self.ctx.check(self.L.hpg_launch_kernel(self.ctx.h, self.pid, KERNEL_CLASSES.index(name), int(precision),
                                                int(reps)), "hpg_launch_kernel")

    def reset_kernel_times(self):
        self.ctx.check(self.L.hpg_reset_kernel_times(self.ctx.h, self.pid))

    # component operators
    def set_state(self, u_full, psi, psi_prev, alpha):
        u, p, pp = _f64(u_full), _f64(psi), _f64(psi_prev)
        self.ctx.check(self.L.hpg_set_state(self.ctx.h, self.pid, _dptr(u), _dptr(p), _dptr(pp), float(alpha)),
                       "hpg_set_state")

    def residual(self):
        F = np.zeros(self.n_u + self.n_psi)
        nrm = C.c_double()
        self.ctx.check(self.L.hpg_residual(self.ctx.h, self.pid, _dptr(F), F.size, C.byref(nrm)), "hpg_residual")
        return F, nrm.value

    def apply_newton(self, x):
        x = _f64(x)
        y = np.zeros_like(x)
        self.ctx.check(self.L.hpg_apply_newton(self.ctx.h, self.pid, _dptr(x), _dptr(y), y.size))
        return y

    def apply_stiffness_inv(self, x, precision=HPG_FP64):
        x = _f64(x)
        y = np.zeros_like(x)
        self.ctx.check(self.L.hpg_apply_stiffness_inv(self.ctx.h, self.pid, int(precision), _dptr(x), _dptr(y),
                                                      y.size))
        return y

    def apply_stiffness_inv_noalloc(self, alpha, x_dev_ptr, y_dev_ptr, length):
        """A_alpha^{-1} on device pointers without any allocation (see hpg.h)."""
        return self.L.hpg_apply_stiffness_inv_noalloc(self.ctx.h, self.pid, float(alpha), C.c_void_p(x_dev_ptr),
                                                       C.c_void_p(y_dev_ptr), int(length))

    def stiffness_solve_pcg(self, b, alpha, rtol=1e-6, atol=1e-6, maxit=2000, precond=3):
        """x = A_alpha^{-1} b by preconditioned CG (precond 1: entity blocks, 2: cell
        patches, 3: vertex-star patches); returns (x, iterations)."""
        b = _f64(b)
        x = np.zeros(self.n_u)
        its = C.c_int()
        self.ctx.check(self.L.hpg_stiffness_solve_pcg(self.ctx.h, self.pid, int(precond), float(alpha), _dptr(b),
                                                      _dptr(x), x.size,
                                                      float(rtol), float(atol), int(maxit), C.byref(its)),
                       "hpg_stiffness_solve_pcg")
        return x, its.value

    def factor_precond(self, precision=HPG_FP64, dump=False):
        if dump:
            # number of cells x nb^2 follows from n_psi (nb = n_psi / cells)
            out = np.zeros(self.n_psi * self._nb())
            self.ctx.check(self.L.hpg_factor_precond(self.ctx.h, self.pid, int(precision), _dptr(out), out.size))
            nb = self._nb()
            return out.reshape(-1, nb, nb)
        self.ctx.check(self.L.hpg_factor_precond(self.ctx.h, self.pid, int(precision), None, 0))
        return None

    def _nb(self):
        return self.n_psi // self.cells

    def apply_precond_inv(self, x, precision=HPG_FP64):
        x = _f64(x)
        y = np.zeros_like(x)
        self.ctx.check(self.L.hpg_apply_precond_inv(self.ctx.h, self.pid, int(precision), _dptr(x), _dptr(y), y.size))
        return y

    def apply_schur(self, x, precision=HPG_FP64):
        x = _f64(x)
        y = np.zeros_like(x)
        self.ctx.check(self.L.hpg_apply_schur(self.ctx.h, self.pid, int(precision), _dptr(x), _dptr(y), y.size))
        return y

    def newton_direction(self, precision=HPG_FP64, rtol=1e-10):
        d = np.zeros(self.n_u + self.n_psi)
        its = C.c_int()
        self.ctx.check(self.L.hpg_newton_direction(self.ctx.h, self.pid, int(precision), float(rtol), _dptr(d),
                                                   d.size, C.byref(its)), "hpg_newton_direction")
        return d, its.value

    # thermoforming QVI (Section 6.4)
    def qvi_points(self, nq=0):
        """Gauss points of the T equation (nq per direction per cell; 0: p + 2)."""
        q = int(nq) if nq else None
        L = self.L
        # the count follows from the cells and nq
        n = self.cells * (q or (self._p + 2)) ** self.dim
        out = np.zeros(n * self.dim)
        self.ctx.check(L.hpg_qvi_points(self.ctx.h, self.pid, int(nq), _dptr(out), out.size), "hpg_qvi_points")
        return out.reshape(n, self.dim)

    def qvi_solve(self, phi0_lat, xi_lat, phi0_q, xi_q, check=True, **kw):
        """Fixed point of the thermoforming QVI; kw sets hpg_qvi_params fields.  Returns
        (status, stats dict)."""
        prm = qvi_default_params(**kw)
        a, b, c, d = (_f64(v) for v in (phi0_lat, xi_lat, phi0_q, xi_q))
        st = hpg_qvi_stats()
        rc = self.L.hpg_qvi_solve(self.ctx.h, self.pid, C.byref(prm), _dptr(a), _dptr(b), min(a.size, b.size),
                                  _dptr(c), _dptr(d), min(c.size, d.size), C.byref(st))
        if check:
            self.ctx.check(rc, "hpg_qvi_solve")
        n = st.iterations
        out = {k: getattr(st, k) for k, _ in hpg_qvi_stats._fields_
               if k not in ("du_h1", "newton_per_fp", "t_newton_per_fp")}
        out["du_h1"] = list(st.du_h1[:n])
        out["newton_per_fp"] = list(st.newton_per_fp[:n])
        out["t_newton_per_fp"] = list(st.t_newton_per_fp[:n])
        return rc, out

    def qvi_T(self):
        out = np.zeros(self.n_u_full)
        self.ctx.check(self.L.hpg_qvi_get_T(self.ctx.h, self.pid, _dptr(out), out.size), "hpg_qvi_get_T")
        return out

    def free(self):
        if self.pid is not None:
            self.L.hpg_problem_free(self.ctx.h, self.pid)
            self.pid = None


def qvi_default_params(**kw):
    prm = hpg_qvi_params()
    lib().hpg_qvi_default_params(C.byref(prm))
    for k, v in kw.items():
        if not hasattr(prm, k):
            raise AttributeError(f"hpg_qvi_params has no field {k}")
        setattr(prm, k, v)
    return prm


def from_workload(ctx, w, params=None):
    """Create and fill a Problem from a ``workloads`` description."""
    bps = w["breakpoints"]
    dim = len(bps)
    lo = [b[0] for b in bps]
    hi = [b[-1] for b in bps]
    cells = [len(b) - 1 for b in bps]
    kind = HPG_GRADIENT if w["kind"] == "gradient" else (HPG_OBSTACLE_LOWER if w.get("lower") else
                                                           HPG_OBSTACLE_UPPER)
    P = Problem(ctx, dim, lo, hi, cells, w["p"], kind)
    if w.get("f_const") is not None:
        P.set_rhs(w["f_const"])
    else:
        P.set_rhs(w["f"])
    P.set_constraint(w["phi"])
    P.set_dirichlet(w.get("g"))
    P.set_alphas(w["alphas"])
    prm = params or default_params()
    prm.beta = w.get("beta", prm.beta)
    prm.newton_tol = w.get("tol", prm.newton_tol)
    P.set_params(prm)
    return P
