"""Python binding of the C ABI in include/tschrod.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert arguments: device arrays are torch tensors (their ``data_ptr()`` is passed),
streams are ``torch.cuda.Stream`` objects (or None for the current stream), and a
non-TS_OK status raises ``TsError`` carrying ``ts_last_error()``.  All computation runs
in the library's CUDA kernels; if the library cannot be loaded, importing this module
fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtschrod.so")

TS_OK, TS_ERR_INVALID_ARG, TS_ERR_NO_MEMORY, TS_ERR_CUDA, TS_ERR_NOT_CONVERGED, TS_ERR_UNSUPPORTED, \
    TS_ERR_TIMEOUT = range(7)
STATUS_NAMES = ["TS_OK", "TS_ERR_INVALID_ARG", "TS_ERR_NO_MEMORY", "TS_ERR_CUDA", "TS_ERR_NOT_CONVERGED",
                "TS_ERR_UNSUPPORTED", "TS_ERR_TIMEOUT"]
TS_FP64, TS_BF16X3, TS_BF16X6, TS_FP32, TS_BF16X1 = 0, 1, 2, 5, 6  # 3 and 4 are not assigned
TS_R64, TS_C128, TS_C64 = range(3)
TS_MAX_DIM = 12

#: Every extern "C" symbol that include/tschrod.h declares.
EXPORTS = [
    "ts_grid_nodes", "ts_tridiag_eig", "ts_plan_create", "ts_plan_destroy", "ts_plan_eigs", "ts_plan_eigvecs", "ts_plan_shape", "ts_plan_bytes",
    "ts_apply_inverse", "ts_apply_inverse_noalloc", "ts_solve_refined", "ts_solve_schedule", "ts_apply_batch", "ts_apply_exp", "ts_apply_operator", "ts_pcg", "ts_inverse_iteration", "ts_split_step",
    "ts_server_create", "ts_server_submit", "ts_server_wait", "ts_server_drain", "ts_server_stats",
    "ts_server_reset_stats", "ts_server_destroy",
    "ts_tc_config_set", "ts_autotune", "ts_device_status", "ts_selftest_wait_timeout", "ts_launch_count", "ts_profile_begin", "ts_profile_end",
    "ts_propagate", "ts_gpe_ground_state", "ts_interpolate", "ts_inverse_iteration_multilevel",
    "ts_last_error", "ts_version",
]


class TsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.POINTER(C.c_int)), ("L", C.POINTER(C.c_double)),
                ("f", C.POINTER(C.POINTER(C.c_double))), ("bc", C.c_int), ("order", C.c_int)]


class _Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("grid", _Desc), ("sigma", C.c_double), ("tau", C.c_double),
                ("V2", C.c_void_p), ("tol", C.c_double), ("maxit", C.c_int), ("in_", C.c_void_p),
                ("out", C.c_void_p), ("dtype", C.c_int), ("prec", C.c_int)]


class _ServerConfig(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_longlong), ("max_inflight", C.c_int), ("max_batch", C.c_int),
                ("plan_cache_entries", C.c_int), ("planner_threads", C.c_int)]


class _ServingStats(C.Structure):
    _fields_ = [("completed", C.c_longlong), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("makespan_ms", C.c_double), ("gdofs", C.c_double), ("plan_hits", C.c_longlong),
                ("plan_misses", C.c_longlong), ("batches", C.c_longlong), ("graph_requests", C.c_longlong),
                ("peak_scratch_bytes", C.c_longlong)]


TS_TC_PAIR = -2  # ts_tc_config_set cluster value: CTA pairs sharing each MMA
TS_SERVER_MAX_INFLIGHT = 1024  # largest ts_server_config.max_inflight
TS_REQ_INVERSE, TS_REQ_EXP, TS_REQ_PCG = range(3)


class _BatchItem(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("dtype", C.c_int), ("prec", C.c_int), ("param", C.c_double),
                ("in_", C.c_void_p), ("out", C.c_void_p)]

_lib = None


def lib() -> C.CDLL:
    """Load libtschrod.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: run `python -m paper_2605_20491_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.c_double, C.c_int
    L.ts_plan_create.argtypes = [C.POINTER(_Desc), C.c_uint, vp, C.POINTER(vp)]
    L.ts_plan_destroy.argtypes = [vp]
    L.ts_plan_eigs.argtypes = [vp, ip, vp]
    L.ts_plan_eigvecs.argtypes = [vp, ip, vp]
    L.ts_plan_shape.argtypes = [vp, C.POINTER(ip), vp, C.POINTER(C.c_longlong)]
    L.ts_plan_bytes.argtypes = [vp, C.POINTER(C.c_longlong)]
    L.ts_apply_inverse.argtypes = [vp, dp, vp, vp, ip, vp]
    L.ts_apply_exp.argtypes = [vp, dp, vp, vp, ip, ip, vp]
    L.ts_solve_refined.argtypes = [vp, dp, vp, vp, ip, ip, vp]
    L.ts_solve_schedule.argtypes = [vp, dp, vp, vp, C.POINTER(ip), ip, vp]
    L.ts_apply_batch.argtypes = [C.POINTER(_BatchItem), ip, vp]
    L.ts_apply_inverse_noalloc.argtypes = [vp, dp, vp, vp, ip, vp]
    L.ts_apply_operator.argtypes = [vp, dp, vp, vp, vp, vp]
    L.ts_pcg.argtypes = [vp, dp, dp, vp, vp, vp, dp, ip, ip, C.POINTER(ip), C.POINTER(dp), vp]
    L.ts_inverse_iteration.argtypes = [vp, dp, vp, vp, ip, dp, ip, dp, ip, ip, C.POINTER(dp), C.POINTER(ip),
                                       C.POINTER(C.c_longlong), vp]
    L.ts_split_step.argtypes = [vp, dp, ip, vp, vp, ip, ip, vp]
    L.ts_propagate.argtypes = [vp, ip, ip, dp, ip, vp, vp, ip, ip, C.POINTER(ip), vp]
    L.ts_grid_nodes.argtypes = [ip, dp, ip, C.POINTER(dp), C.POINTER(dp)]
    L.ts_tridiag_eig.argtypes = [ip, C.POINTER(dp), C.POINTER(dp), C.POINTER(dp), C.POINTER(dp)]
    L.ts_interpolate.argtypes = [vp, vp, vp, vp, vp]
    L.ts_inverse_iteration_multilevel.argtypes = [C.POINTER(vp), C.POINTER(vp), ip, dp, vp, dp, ip, dp, ip, ip,
                                                  C.POINTER(dp), C.POINTER(ip), C.POINTER(C.c_longlong), vp]
    L.ts_gpe_ground_state.argtypes = [vp, vp, dp, ip, dp, dp, vp, dp, dp, ip, ip, dp, C.POINTER(dp), C.POINTER(dp),
                                      C.POINTER(dp), C.POINTER(ip), C.POINTER(C.c_longlong), vp]
    L.ts_device_status.argtypes = [vp]
    L.ts_selftest_wait_timeout.argtypes = [C.c_longlong, vp]
    L.ts_server_create.argtypes = [C.POINTER(_ServerConfig), C.POINTER(vp)]
    L.ts_server_submit.argtypes = [vp, C.POINTER(_Request), C.POINTER(C.c_longlong)]
    L.ts_server_wait.argtypes = [vp, C.c_longlong, C.POINTER(ip), C.POINTER(dp), C.POINTER(ip)]
    L.ts_server_drain.argtypes = [vp]
    L.ts_server_stats.argtypes = [vp, C.POINTER(_ServingStats)]
    L.ts_server_reset_stats.argtypes = [vp]
    L.ts_server_destroy.argtypes = [vp]
    L.ts_tc_config_set.argtypes = [ip, ip, ip, ip, ip]
    L.ts_autotune.argtypes = [vp, ip, ip, C.c_char_p, C.POINTER(ip), vp]
    L.ts_launch_count.argtypes = []
    L.ts_profile_begin.argtypes = []
    L.ts_profile_end.argtypes = [ip, C.POINTER(C.c_longlong), C.POINTER(dp), C.POINTER(dp), C.POINTER(dp)]
    L.ts_last_error.restype = C.c_char_p
    L.ts_last_error.argtypes = []
    L.ts_version.restype = C.c_char_p
    L.ts_version.argtypes = []
    for name in EXPORTS:
        if name not in ("ts_last_error", "ts_version"):
            getattr(L, name).restype = C.c_int
    L.ts_launch_count.restype = C.c_longlong
    _lib = L
    return L


def ts_last_error() -> str:
    return lib().ts_last_error().decode()


def ts_version() -> str:
    return lib().ts_version().decode()


def _check(status: int, where: str, allow=()):
    if status != TS_OK and status not in allow:
        raise TsError(status, where, ts_last_error())
    return status


def _ptr(t) -> C.c_void_p | None:
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Plan:
    """Owning handle of a ts_plan (freed by ts_plan_destroy on close / garbage collection)."""

    def __init__(self, handle: int, n, L):
        self.handle = C.c_void_p(handle)
        self.n = tuple(n)
        self.L = tuple(L)
        self.N = int(np.prod(self.n))

    @property
    def d(self) -> int:
        return len(self.n)

    def close(self):
        ts_plan_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ts_grid_nodes(n: int, L: float, order: int = 1):
    """Interior nodes and lumped masses of one axis: (x, m), n doubles each (host)."""
    x, m = np.empty(int(n)), np.empty(int(n))
    _check(lib().ts_grid_nodes(C.c_int(int(n)), C.c_double(float(L)), C.c_int(int(order)),
                               x.ctypes.data_as(C.POINTER(C.c_double)), m.ctypes.data_as(C.POINTER(C.c_double))),
           "ts_grid_nodes")
    return x, m


def ts_tridiag_eig(diag, offdiag):
    """Eigenvalues (ascending) and unit eigenvectors (columns) of the symmetric tridiagonal
    matrix with this diagonal and off-diagonal, on the host: (lam, Z) with T = Z diag(lam) Z^T."""
    a = np.ascontiguousarray(np.asarray(diag, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(offdiag, dtype=np.float64))
    n = a.size
    lam, Zc = np.empty(n), np.empty((n, n))  # Zc[j] = eigenvector j (column-major Z)
    P = C.POINTER(C.c_double)
    _check(lib().ts_tridiag_eig(C.c_int(n), a.ctypes.data_as(P), b.ctypes.data_as(P) if b.size else None,
                                lam.ctypes.data_as(P), Zc.ctypes.data_as(P)), "ts_tridiag_eig")
    return lam, Zc.T.copy()


def ts_plan_create(n, L, f, precision_mask: int = 0, stream=None, bc: int = 0, order: int = 1) -> Plan:
    """order = k of Q^k (1: finite differences on uniform nodes; >= 2: spectral elements,
    f sampled at ts_grid_nodes(n_k, L_k, order))."""
    d = len(n)
    f_arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in f]
    n_arr = (C.c_int * d)(*[int(v) for v in n])
    L_arr = (C.c_double * d)(*[float(v) for v in L])
    f_ptrs = (C.POINTER(C.c_double) * d)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in f_arrs])
    desc = _Desc(d, n_arr, L_arr, f_ptrs, bc, order)
    out = C.c_void_p()
    _check(lib().ts_plan_create(C.byref(desc), precision_mask, _stream(stream), C.byref(out)), "ts_plan_create")
    return Plan(out.value, n, L)


def ts_plan_destroy(plan: Plan):
    """Frees the plan once: the handle is cleared first, so a later close() or garbage
    collection of the same object does nothing.  The device is synchronised first, since a
    Python object may be collected while kernels that read its tables are still queued."""
    h, plan.handle = plan.handle, C.c_void_p(None)
    if h:
        import torch
        if torch.cuda.is_initialized():
            torch.cuda.synchronize()
        _check(lib().ts_plan_destroy(h), "ts_plan_destroy")


def ts_plan_eigs(plan: Plan, axis: int) -> np.ndarray:
    out = np.empty(plan.n[axis])
    _check(lib().ts_plan_eigs(plan.handle, axis, out.ctypes.data), "ts_plan_eigs")
    return out


def ts_plan_eigvecs(plan: Plan, axis: int) -> np.ndarray:
    out = np.empty((plan.n[axis], plan.n[axis]))
    _check(lib().ts_plan_eigvecs(plan.handle, axis, out.ctypes.data), "ts_plan_eigvecs")
    return out


def ts_plan_bytes(plan: Plan) -> int:
    v = C.c_longlong()
    _check(lib().ts_plan_bytes(plan.handle, C.byref(v)), "ts_plan_bytes")
    return v.value


def ts_apply_inverse(plan: Plan, sigma: float, b, u, prec: int = TS_FP64, stream=None):
    _check(lib().ts_apply_inverse(plan.handle, sigma, _ptr(b), _ptr(u), prec, _stream(stream)), "ts_apply_inverse")


def ts_apply_inverse_noalloc(plan: Plan, sigma: float, b, u, prec: int = TS_FP64, stream=None):
    """ts_apply_inverse with its work buffers in a fixed 32 MiB array inside the library,
    for callers that must not allocate device memory (see include/tschrod.h)."""
    _check(lib().ts_apply_inverse_noalloc(plan.handle, sigma, _ptr(b), _ptr(u), prec, _stream(stream)),
           "ts_apply_inverse_noalloc")


def ts_solve_refined(plan: Plan, sigma: float, b, u, prec: int = TS_BF16X3, refinements: int = 2, stream=None):
    _check(lib().ts_solve_refined(plan.handle, sigma, _ptr(b), _ptr(u), prec, refinements, _stream(stream)),
           "ts_solve_refined")


def ts_solve_schedule(plan: Plan, sigma: float, b, u, schedule, stream=None):
    """u_0 = P_0 b, then one refinement per further entry of `schedule` (precisions)."""
    arr = (C.c_int * len(schedule))(*schedule)
    _check(lib().ts_solve_schedule(plan.handle, sigma, _ptr(b), _ptr(u), arr, len(schedule), _stream(stream)),
           "ts_solve_schedule")


def ts_apply_batch(items, stream=None):
    """items: (plan, dtype, prec, param, in, out) tuples; TS_R64 = inverse (param sigma),
    TS_C128 / TS_C64 = exp (param tau).  One launch per stage over all items."""
    arr = (_BatchItem * max(1, len(items)))()
    for k, (plan, dtype, prec, param, xin, xout) in enumerate(items):
        arr[k] = _BatchItem(plan.handle, dtype, prec, param, _ptr(xin), _ptr(xout))
    _check(lib().ts_apply_batch(arr, len(items), _stream(stream)), "ts_apply_batch")


def ts_apply_exp(plan: Plan, tau: float, psi_in, psi_out, dtype: int, prec: int = TS_FP64, stream=None):
    _check(lib().ts_apply_exp(plan.handle, tau, _ptr(psi_in), _ptr(psi_out), dtype, prec, _stream(stream)),
           "ts_apply_exp")


def ts_apply_operator(plan: Plan, sigma: float, V2, x, y, stream=None):
    _check(lib().ts_apply_operator(plan.handle, sigma, _ptr(V2), _ptr(x), _ptr(y), _stream(stream)),
           "ts_apply_operator")


def ts_pcg(plan: Plan, sigma: float, sigma_P: float, V2, b, x, tol: float, maxit: int, precond: int = TS_FP64,
           stream=None, allow_not_converged: bool = False):
    """Returns (status, iterations, true relative residual)."""
    it = C.c_int(0)
    rel = C.c_double(0.0)
    st = lib().ts_pcg(plan.handle, sigma, sigma_P, _ptr(V2), _ptr(b), _ptr(x), tol, maxit, precond,
                      C.byref(it), C.byref(rel), _stream(stream))
    _check(st, "ts_pcg", allow=(TS_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, it.value, rel.value


def ts_inverse_iteration(plan: Plan, shift: float, V2, u, init_from_plan: bool = True, tol_lambda: float = 1e-12,
                         maxit: int = 200, pcg_tol: float = 1e-10, pcg_maxit: int = 500, precond: int = TS_FP64,
                         stream=None):
    """Returns (lambda, outer iterations, total PCG iterations)."""
    lam = C.c_double(0.0)
    outer = C.c_int(0)
    tot = C.c_longlong(0)
    _check(lib().ts_inverse_iteration(plan.handle, shift, _ptr(V2), _ptr(u), int(init_from_plan), tol_lambda, maxit,
                                      pcg_tol, pcg_maxit, precond, C.byref(lam), C.byref(outer), C.byref(tot),
                                      _stream(stream)), "ts_inverse_iteration")
    return lam.value, outer.value, tot.value


def ts_tc_config_set(complex_data: bool, n: int, bk: int, bn_cap: int, cluster: int = 1):
    _check(lib().ts_tc_config_set(int(complex_data), n, bk, bn_cap, cluster), "ts_tc_config_set")


def ts_tc_config_reset(complex_data: bool, n: int = 0):
    """Forget the tile configuration for (complex_data, n): the built-in choice applies again."""
    _check(lib().ts_tc_config_set(int(complex_data), n, 0, 0, 0), "ts_tc_config_set")


def ts_autotune(plan: Plan, dtype: int, prec: int, cache_path: str | None = None, stream=None) -> int:
    """Returns the number of axis lengths that were searched (0 = all from the cache)."""
    tuned = C.c_int(0)
    path = cache_path.encode() if cache_path else None
    _check(lib().ts_autotune(plan.handle, dtype, prec, path, C.byref(tuned), _stream(stream)), "ts_autotune")
    return tuned.value


def ts_selftest_wait_timeout(cycles: int, stream=None):
    _check(lib().ts_selftest_wait_timeout(cycles, _stream(stream)), "ts_selftest_wait_timeout")


def ts_launch_count() -> int:
    return lib().ts_launch_count()


def ts_profile_begin():
    _check(lib().ts_profile_begin(), "ts_profile_begin")


PROF_TC_PASS, PROF_FP64_PASS, PROF_SMALL_PASS, PROF_RESIDUAL, PROF_TC_PASS_X1, PROF_TC_PASS_OUT, PROF_TC_LIST = range(7)


def ts_profile_end(kind: int):
    """Returns (launches, total ms, algorithmic FLOPs, algorithmic bytes) for one kernel kind."""
    n = C.c_longlong(0)
    ms, fl, by = C.c_double(0), C.c_double(0), C.c_double(0)
    _check(lib().ts_profile_end(kind, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)), "ts_profile_end")
    return n.value, ms.value, fl.value, by.value


def ts_device_status(stream=None):
    _check(lib().ts_device_status(_stream(stream)), "ts_device_status")


def ts_split_step(plan: Plan, dt: float, nsteps: int, V2, psi, dtype: int, prec: int = TS_FP64, stream=None):
    _check(lib().ts_split_step(plan.handle, dt, nsteps, _ptr(V2), _ptr(psi), dtype, prec, _stream(stream)),
           "ts_split_step")


TS_STRANG, TS_QHOP, TS_MAGNUS2 = range(3)


def ts_propagate(plan: Plan, scheme: int, M: int, dt: float, nsteps: int, VB, psi, dtype: int, prec: int = TS_FP64,
                 stream=None) -> int:
    """Splitting steps of Sec. 5.1 in place on psi; returns the number of A-propagations."""
    na = C.c_int(0)
    _check(lib().ts_propagate(plan.handle, int(scheme), int(M), float(dt), int(nsteps), _ptr(VB), _ptr(psi), dtype,
                              prec, C.byref(na), _stream(stream)), "ts_propagate")
    return na.value


def ts_interpolate(coarse: Plan, uc, fine: Plan, uf, stream=None):
    _check(lib().ts_interpolate(coarse.handle, _ptr(uc), fine.handle, _ptr(uf), _stream(stream)), "ts_interpolate")


def ts_inverse_iteration_multilevel(plans, V2s, shift: float, u, tol_lambda: float = 1e-12, maxit: int = 200,
                                    pcg_tol: float = 1e-12, pcg_maxit: int = 500, precond: int = TS_FP64,
                                    stream=None):
    """Returns (lambda, [outer iterations per level], [PCG iterations per level]); u (finest
    grid) receives the eigenvector."""
    lv = len(plans)
    P = (C.c_void_p * lv)(*[p.handle.value if isinstance(p.handle, C.c_void_p) else p.handle for p in plans])
    V = (C.c_void_p * lv)(*[None if v is None else v.data_ptr() for v in (V2s if V2s is not None else [None] * lv)])
    lam = C.c_double()
    outer = (C.c_int * lv)()
    pcg = (C.c_longlong * lv)()
    _check(lib().ts_inverse_iteration_multilevel(P, V, lv, float(shift), _ptr(u), float(tol_lambda), int(maxit),
                                                 float(pcg_tol), int(pcg_maxit), int(precond), C.byref(lam), outer,
                                                 pcg, _stream(stream)), "ts_inverse_iteration_multilevel")
    return lam.value, list(outer), list(pcg)


TS_GPE_H1, TS_GPE_AU = range(2)


def ts_gpe_ground_state(plan: Plan, V2, beta: float, flow: int, u, alpha: float = 20.0, tau: float = 0.1,
                        tol_energy: float = 1e-14, tol_residual: float = 0.0, maxit: int = 5000, prec: int = TS_FP64,
                        pcg_tol: float = 1e-12, stream=None, allow_not_converged: bool = False):
    """Returns (energy, lambda, iterations, solves, residual); u is updated in place."""
    E, lam, res, it, so = C.c_double(), C.c_double(), C.c_double(), C.c_int(), C.c_longlong()
    st = lib().ts_gpe_ground_state(plan.handle, _ptr(V2), float(beta), int(flow), float(alpha), float(tau), _ptr(u),
                                   float(tol_energy), float(tol_residual), int(maxit), int(prec), float(pcg_tol),
                                   C.byref(E), C.byref(lam), C.byref(res), C.byref(it), C.byref(so), _stream(stream))
    _check(st, "ts_gpe_ground_state", allow=(TS_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return E.value, lam.value, it.value, so.value, res.value


class Server:
    """Owning handle of a ts_server.  Keeps every submitted request's arguments alive until
    it has been waited for."""

    def __init__(self, memory_budget_bytes: int = 0, max_inflight: int = 8, max_batch: int = 0,
                 plan_cache_entries: int = 1024, planner_threads: int = 0):
        cfg = _ServerConfig(memory_budget_bytes, max_inflight, max_batch, plan_cache_entries, planner_threads)
        h = C.c_void_p()
        _check(lib().ts_server_create(C.byref(cfg), C.byref(h)), "ts_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, kind: int, n, L, f, inp, out, sigma: float = 0.0, tau: float = 0.0, V2=None, tol: float = 1e-10,
               maxit: int = 200, dtype: int = TS_R64, prec: int = TS_FP64, order: int = 1) -> int:
        d = len(n)
        f_arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in f]
        n_arr = (C.c_int * d)(*[int(v) for v in n])
        L_arr = (C.c_double * d)(*[float(v) for v in L])
        f_ptrs = (C.POINTER(C.c_double) * d)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in f_arrs])
        req = _Request(kind, _Desc(d, n_arr, L_arr, f_ptrs, 0, order), sigma, tau, _ptr(V2), tol, maxit, _ptr(inp),
                       _ptr(out), dtype, prec)
        ticket = C.c_longlong()
        _check(lib().ts_server_submit(self.handle, C.byref(req), C.byref(ticket)), "ts_server_submit")
        self._keep[ticket.value] = (inp, out, V2)
        return ticket.value

    def wait(self, ticket: int):
        """Returns (status, latency_ms, iterations)."""
        st, lat, it = C.c_int(), C.c_double(), C.c_int()
        _check(lib().ts_server_wait(self.handle, ticket, C.byref(st), C.byref(lat), C.byref(it)), "ts_server_wait")
        self._keep.pop(ticket, None)
        return st.value, lat.value, it.value

    def drain(self):
        _check(lib().ts_server_drain(self.handle), "ts_server_drain")

    def stats(self) -> dict:
        s = _ServingStats()
        _check(lib().ts_server_stats(self.handle, C.byref(s)), "ts_server_stats")
        return {k: getattr(s, k) for k, _ in _ServingStats._fields_}

    def reset_stats(self):
        _check(lib().ts_server_reset_stats(self.handle), "ts_server_reset_stats")

    def close(self):
        if self.handle:
            _check(lib().ts_server_destroy(self.handle), "ts_server_destroy")
            self.handle = C.c_void_p(None)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
