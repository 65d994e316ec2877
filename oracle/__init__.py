"""CPU FP64 oracle of the tensor-product Schroedinger solver (ctypes binding of oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark are the only users.  The library product never imports this package,
and this package never imports the library.

Each function below is a thin marshalling layer over the C function of the same name
in ``oracle.c``, whose header cites the passage of the paper that it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"])
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_grid.argtypes = [C.c_int, C.c_double, _dp]
        L.or_operator_1d.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.or_jacobi_eigh.argtypes = [C.c_int, _dp, _dp, _dp]
        L.or_jacobi_eigh.restype = C.c_int
        L.or_mode_forward.argtypes = [C.c_int, _ip, C.c_int, _dp, C.c_int, _dp, _dp]
        L.or_mode_backward.argtypes = [C.c_int, _ip, C.c_int, _dp, C.c_int, _dp, _dp]
        L.or_mode_fibers.argtypes = [C.c_int, _ip, C.c_int, _dp, C.c_int, _dp, _dp, C.c_long, C.c_long]
        L.or_apply_inverse.argtypes = [C.c_int, _ip, C.POINTER(_dp), C.POINTER(_dp), C.c_double, _dp, _dp]
        L.or_apply_exp.argtypes = [C.c_int, _ip, C.POINTER(_dp), C.POINTER(_dp), C.c_double, _dp, _dp]
        L.or_dense_operator.argtypes = [C.c_int, _ip, C.POINTER(_dp), _dp, C.c_double, _dp]
        L.or_lu_solve.argtypes = [C.c_long, _dp, _dp, _dp]
        L.or_lu_solve.restype = C.c_int
        L.or_dense_exp.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp]
        L.or_dense_exp.restype = C.c_int
        L.or_stencil.argtypes = [C.c_int, _ip, _dp, C.POINTER(_dp), _dp, C.c_double, _dp, _dp]
        L.or_pcg.argtypes = [C.c_int, _ip, _dp, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp), _dp,
                             C.c_double, C.c_double, _dp, _dp, C.c_double, C.c_int, _dp]
        L.or_pcg.restype = C.c_int
        L.or_inverse_iteration.argtypes = [C.c_int, _ip, _dp, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp),
                                           _dp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                                           _dp, _dp, C.POINTER(C.c_long)]
        L.or_inverse_iteration.restype = C.c_int
        L.or_strang.argtypes = [C.c_int, _ip, C.POINTER(_dp), C.POINTER(_dp), _dp, C.c_double, C.c_int, _dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr_array(arrs):
    return (_dp * len(arrs))(*[_p(a) for a in arrs])


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(t: int) -> None:
    lib().or_set_num_threads(int(t))


def grid(n: int, L: float) -> np.ndarray:
    x = np.empty(n)
    lib().or_grid(n, L, _p(x))
    return x


def operator_1d(n: int, L: float, f) -> np.ndarray:
    H = np.empty((n, n))
    lib().or_operator_1d(n, L, _p(_f64(f)), _p(H))
    return H


def jacobi_eigh(A):
    A = _f64(A)
    n = A.shape[0]
    lam = np.empty(n)
    Q = np.empty((n, n))
    sweeps = lib().or_jacobi_eigh(n, _p(A), _p(lam), _p(Q))
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    return lam, Q


@dataclass
class Plan:
    """Per-axis data of the separable operator: sizes n_k, half-widths L_k, sampled
    f_k, and the eigendecompositions H_k = S_k diag(lam_k) S_k^T (step 1 of Sec. 2.1)."""
    n: tuple
    L: tuple
    f: list
    S: list = field(default_factory=list)
    lam: list = field(default_factory=list)

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def _n(self):
        return (C.c_int * self.d)(*self.n)


def plan(n, L, f) -> Plan:
    n = tuple(int(v) for v in n)
    L = tuple(float(v) for v in L)
    f = [_f64(v) for v in f]
    P = Plan(n, L, f)
    for k in range(len(n)):
        lam, S = jacobi_eigh(operator_1d(n[k], L[k], f[k]))
        P.S.append(_f64(S))
        P.lam.append(_f64(lam))
    return P


def mode_forward(P: Plan, k: int, X, ncomp: int = 1) -> np.ndarray:
    X = _f64(X)
    Y = np.empty_like(X)
    lib().or_mode_forward(P.d, P._n(), k, _p(P.S[k]), ncomp, _p(X), _p(Y))
    return Y


def mode_backward(P: Plan, k: int, X, ncomp: int = 1) -> np.ndarray:
    X = _f64(X)
    Y = np.empty_like(X)
    lib().or_mode_backward(P.d, P._n(), k, _p(P.S[k]), ncomp, _p(X), _p(Y))
    return Y


def mode_fibers(P: Plan, k: int, X, Y, backward: bool, f0: int, f1: int) -> None:
    """Timing sample: the forward (or backward) transform along axis k of real X, written
    into Y, for the fibers with flat index in [f0, f1) only (see or_mode_fibers)."""
    lib().or_mode_fibers(P.d, P._n(), k, _p(P.S[k]), int(backward), _p(X), _p(Y), int(f0), int(f1))


def apply_inverse(P: Plan, sigma: float, b) -> np.ndarray:
    b = _f64(b)
    u = np.empty_like(b)
    lib().or_apply_inverse(P.d, P._n(), _ptr_array(P.S), _ptr_array(P.lam), sigma, _p(b), _p(u))
    return u


def apply_exp(P: Plan, tau: float, psi) -> np.ndarray:
    """psi: complex interleaved float64 of length 2N."""
    psi = _f64(psi)
    out = np.empty_like(psi)
    lib().or_apply_exp(P.d, P._n(), _ptr_array(P.S), _ptr_array(P.lam), tau, _p(psi), _p(out))
    return out


def dense_operator(P: Plan, sigma: float = 0.0, V2=None) -> np.ndarray:
    H = [operator_1d(P.n[k], P.L[k], P.f[k]) for k in range(P.d)]
    A = np.empty((P.N, P.N))
    v2 = _p(_f64(V2)) if V2 is not None else None
    lib().or_dense_operator(P.d, P._n(), _ptr_array(H), v2, sigma, _p(A))
    return A


def lu_solve(A, b) -> np.ndarray:
    A = _f64(A)
    b = _f64(b)
    x = np.empty_like(b)
    if lib().or_lu_solve(A.shape[0], _p(A), _p(b), _p(x)) != 0:
        raise RuntimeError("singular matrix")
    return x


def dense_exp(H, tau: float, psi) -> np.ndarray:
    H = _f64(H)
    psi = _f64(psi)
    out = np.empty_like(psi)
    if lib().or_dense_exp(H.shape[0], _p(H), tau, _p(psi), _p(out)) < 0:
        raise RuntimeError("Jacobi did not converge")
    return out


def stencil(P: Plan, x, sigma: float = 0.0, V2=None) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    v2 = _p(_f64(V2)) if V2 is not None else None
    lib().or_stencil(P.d, P._n(), _p(_f64(P.L)), _ptr_array(P.f), v2, sigma, _p(x), _p(y))
    return y


def pcg(P: Plan, b, sigma: float = 0.0, sigma_P: float | None = None, V2=None, x0=None,
        tol: float = 1e-10, maxit: int = 500):
    """Returns (x, iterations, true relative residual); iterations < 0 if maxit was hit."""
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    sigma_P = sigma if sigma_P is None else sigma_P
    rel = C.c_double(0.0)
    v2 = _p(_f64(V2)) if V2 is not None else None
    it = lib().or_pcg(P.d, P._n(), _p(_f64(P.L)), _ptr_array(P.f), _ptr_array(P.S), _ptr_array(P.lam),
                      v2, sigma, sigma_P, _p(b), _p(x), tol, maxit, C.byref(rel))
    return x, it, rel.value


def inverse_iteration(P: Plan, shift: float, V2=None, tol_lambda: float = 1e-12, maxit: int = 200,
                      pcg_tol: float = 1e-10, pcg_maxit: int = 500):
    """Returns (u, lambda, outer iterations, total PCG iterations)."""
    u = np.empty(P.N)
    lam = C.c_double(0.0)
    tot = C.c_long(0)
    v2 = _p(_f64(V2)) if V2 is not None else None
    it = lib().or_inverse_iteration(P.d, P._n(), _p(_f64(P.L)), _ptr_array(P.f), _ptr_array(P.S),
                                    _ptr_array(P.lam), v2, shift, tol_lambda, maxit, pcg_tol, pcg_maxit,
                                    _p(u), C.byref(lam), C.byref(tot))
    return u, lam.value, it, tot.value


def strang(P: Plan, V2, dt: float, nsteps: int, psi) -> np.ndarray:
    psi = _f64(psi).copy()
    lib().or_strang(P.d, P._n(), _ptr_array(P.S), _ptr_array(P.lam), _p(_f64(V2)), dt, nsteps, _p(psi))
    return psi
