"""CPU FP64 oracle of the Q^k spectral element discretisation (k >= 1) and of the
tensor-product solver built on it.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark are the only users.  The library product never imports this module, and
this module never imports the library.  It is plain numpy in FP64: library primitives
(Legendre polynomials, a small linear solve, a symmetric eigensolver, tensordot) serve as
steps; there is no blocking, fusion or reordering beyond what the definitions state.

What it computes (Sec. 2, eqs. general_system, tensor_system, eigen_decomp):

* Per axis, [-L, L] is cut into c elements of width h_e = 2L / c.  Each element carries the
  k + 1 Gauss-Lobatto-Legendre (GLL) points of degree k mapped onto it; neighbouring
  elements share their end points, so there are c k + 1 nodes, and the c k - 1 interior
  ones carry the unknowns (homogeneous Dirichlet): n = c k - 1.
* Every integral is evaluated by the (k + 1)-point GLL rule, so the mass matrix M is
  diagonal (m_i = sum over elements holding node i of (h_e / 2) w_q), the potential term
  is M diag(V(x_i)) and the load is M f(x_i).  The stiffness matrix is
  Stiff_ij = sum_e (2 / h_e) sum_q w_q l_i'(xi_q) l_j'(xi_q).
* The 1D discrete Laplacian is K = M^{-1} Stiff and H = K + diag f.  H is similar to the
  symmetric M^{-1/2} Stiff M^{-1/2} + diag f = Q Lambda Q^T, so H = T Lambda T^{-1} with
  T = M^{-1/2} Q and T^{-1} = Q^T M^{1/2} (eq. eigen_decomp).
* The d-dimensional operator is A = sum_k (I x .. x H_k x .. x I) + diag(V2) + sigma I; the
  direct solve and the propagator are the 4 steps of Sec. 2.1 with T_k^{-1} forward and T_k
  backward.

For k = 1 this is the second-order finite-difference scheme of the other oracle
(K = h^-2 tridiag(-1, 2, -1), uniform nodes).

Array convention: vec(X), axis 1 fastest, i.e. a numpy array of shape (n_d, ..., n_1) in
C order, flattened.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------- reference element -----

def gll(k: int):
    """GLL points and weights of degree k on [-1, 1] (k + 1 points): the end points and
    the roots of P_k'; w_j = 2 / (k (k + 1) P_k(xi_j)^2)."""
    if k < 1:
        raise ValueError("k >= 1")
    Pk = npleg.Legendre.basis(k)
    inner = np.sort(np.real(Pk.deriv().roots())) if k >= 2 else np.zeros(0)
    xi = np.concatenate(([-1.0], inner, [1.0]))
    w = 2.0 / (k * (k + 1) * Pk(xi) ** 2)
    return xi, w


def diff_matrix(xi) -> np.ndarray:
    """D[q][j] = l_j'(xi_q) for the Lagrange basis l_j of the nodes xi.  The basis is
    written in Legendre polynomials: V[q][m] = P_m(xi_q), l_j = sum_m C[m][j] P_m with
    V C = I, so D = V' C with V'[q][m] = P_m'(xi_q)."""
    xi = np.asarray(xi, dtype=np.float64)
    k = len(xi) - 1
    V = npleg.legvander(xi, k)
    Vd = np.zeros_like(V)
    for m in range(k + 1):
        Vd[:, m] = npleg.legval(xi, npleg.legder(np.eye(k + 1)[m]))
    C = np.linalg.solve(V, np.eye(k + 1))
    return Vd @ C


def element_matrices(k: int, h: float):
    """Stiffness and lumped mass of one element of width h:
    Se[i][j] = (2 / h) sum_q w_q D[q][i] D[q][j],  me[q] = (h / 2) w_q."""
    xi, w = gll(k)
    D = diff_matrix(xi)
    Se = (2.0 / h) * (D.T * w) @ D
    return Se, 0.5 * h * w


# ----------------------------------------------------------------------- one axis --------

@dataclass
class Axis1D:
    k: int
    L: float
    x: np.ndarray      # interior node coordinates, n
    m: np.ndarray      # lumped mass, n
    stiff: np.ndarray  # n x n


def cells(n: int, k: int) -> int:
    if (n + 1) % k:
        raise ValueError(f"Q^{k}: n + 1 = {n + 1} is not a multiple of k")
    return (n + 1) // k


def axis_1d(n: int, L: float, k: int) -> Axis1D:
    """Nodes, lumped mass and stiffness of one axis, assembled over the c = (n+1)/k
    elements and restricted to the interior nodes."""
    c = cells(n, k)
    he = 2.0 * L / c
    xi, _ = gll(k)
    Se, me = element_matrices(k, he)
    G = c * k + 1
    S = np.zeros((G, G))
    m = np.zeros(G)
    x = np.zeros(G)
    for e in range(c):
        g = e * k + np.arange(k + 1)
        S[np.ix_(g, g)] += Se
        m[g] += me
        x[g] = -L + e * he + 0.5 * (xi + 1.0) * he
    return Axis1D(k, L, x[1:-1].copy(), m[1:-1].copy(), S[1:-1, 1:-1].copy())


def laplacian_1d(ax: Axis1D) -> np.ndarray:
    """K = M^{-1} Stiff (not symmetric for k >= 2)."""
    return ax.stiff / ax.m[:, None]


# ------------------------------------------------------------------------- plan -----------

@dataclass
class SemPlan:
    n: tuple
    L: tuple
    k: int
    axes: list = field(default_factory=list)
    f: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    Q: list = field(default_factory=list)     # eigenvectors of the symmetric form (columns)
    T: list = field(default_factory=list)     # M^{-1/2} Q
    Tinv: list = field(default_factory=list)  # Q^T M^{1/2}

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def shape(self):
        return tuple(reversed(self.n))


def plan(n, L, f, k: int) -> SemPlan:
    """Step 1 of Sec. 2.1 for Q^k: per axis, eigendecompose M^{-1/2} Stiff M^{-1/2} + diag f
    (f sampled at the interior nodes) and form T, T^{-1} (eq. eigen_decomp)."""
    n = tuple(int(v) for v in n)
    L = tuple(float(v) for v in (L if np.ndim(L) else [L] * len(n)))
    P = SemPlan(n, L, k)
    for a in range(len(n)):
        ax = axis_1d(n[a], L[a], k)
        fa = np.asarray(f[a], dtype=np.float64)
        r = 1.0 / np.sqrt(ax.m)
        Hs = r[:, None] * ax.stiff * r[None, :] + np.diag(fa)
        Hs = 0.5 * (Hs + Hs.T)
        lam, Q = np.linalg.eigh(Hs)
        P.axes.append(ax)
        P.f.append(fa)
        P.lam.append(lam)
        P.Q.append(Q)
        P.T.append(r[:, None] * Q)
        P.Tinv.append(Q.T * np.sqrt(ax.m)[None, :])
    return P


def nodes(P: SemPlan, a: int) -> np.ndarray:
    return P.axes[a].x


def along(P: SemPlan, a: int, A, X) -> np.ndarray:
    """Y[.., i, ..] = sum_j A[i][j] X[.., j, ..] along axis a (axis 1 is the last numpy axis)."""
    ax = P.d - 1 - a
    Y = np.tensordot(A, X, axes=([1], [ax]))
    return np.moveaxis(Y, 0, ax)


def lambda_sum(P: SemPlan) -> np.ndarray:
    """Lambda_idx = sum_k lambda_{k, i_k} as an array of the grid's shape."""
    S = np.zeros(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        S = S + P.lam[a].reshape(sh)
    return S


def potential_sum(P: SemPlan) -> np.ndarray:
    """V1 at the grid nodes, sum_k f_k(x_{k, i_k})."""
    S = np.zeros(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        S = S + P.f[a].reshape(sh)
    return S


def mass_product(P: SemPlan) -> np.ndarray:
    """The d-dimensional lumped mass prod_k m_{k, i_k} (the M of the M-inner product)."""
    S = np.ones(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        S = S * P.axes[a].m.reshape(sh)
    return S


def apply_inverse(P: SemPlan, sigma: float, b) -> np.ndarray:
    """u = (A + sigma)^{-1} b by steps 2-4 of Sec. 2.1: T^{-1} on every axis, divide by the
    eigenvalue sums plus sigma, T on every axis."""
    X = np.asarray(b, dtype=np.float64).reshape(P.shape())
    for a in range(P.d):
        X = along(P, a, P.Tinv[a], X)
    X = X / (lambda_sum(P) + sigma)
    for a in range(P.d):
        X = along(P, a, P.T[a], X)
    return X.reshape(-1)


def apply_exp(P: SemPlan, tau: float, psi) -> np.ndarray:
    """e^{-i tau A} psi = T (e^{-i tau Lambda} . T^{-1} psi) (Sec. 2.1), psi complex."""
    X = np.asarray(psi, dtype=np.complex128).reshape(P.shape())
    for a in range(P.d):
        X = along(P, a, P.Tinv[a], X)
    X = X * np.exp(-1j * tau * lambda_sum(P))
    for a in range(P.d):
        X = along(P, a, P.T[a], X)
    return X.reshape(-1)


def operator(P: SemPlan, x, sigma: float = 0.0, V2=None) -> np.ndarray:
    """A x = sum_k K_k x along axis k + (V1 + V2 + sigma) x, K_k = M_k^{-1} Stiff_k
    (eq. general_system with the Q^k Laplacian)."""
    X = np.asarray(x, dtype=np.float64).reshape(P.shape())
    Y = (potential_sum(P) + sigma) * X
    if V2 is not None:
        Y = Y + np.asarray(V2, dtype=np.float64).reshape(P.shape()) * X
    for a in range(P.d):
        Y = Y + along(P, a, laplacian_1d(P.axes[a]), X)
    return Y.reshape(-1)


def dense_operator(P: SemPlan, sigma: float = 0.0, V2=None) -> np.ndarray:
    """The N x N matrix of eq. general_system as a Kronecker sum (small N only)."""
    N = P.N
    A = np.zeros((N, N))
    for a in range(P.d):
        Ka = laplacian_1d(P.axes[a]) + np.diag(P.f[a])
        left = int(np.prod(P.n[a + 1:])) if a + 1 < P.d else 1
        right = int(np.prod(P.n[:a])) if a > 0 else 1
        A += np.kron(np.eye(left), np.kron(Ka, np.eye(right)))
    A += sigma * np.eye(N)
    if V2 is not None:
        A += np.diag(np.asarray(V2, dtype=np.float64).reshape(-1))
    return A


# ------------------------------------------------------------------- iterative -----------

def _mdot(W, a, b) -> float:
    return float(np.sum(W * a * b))


def pcg(P: SemPlan, b, sigma: float = 0.0, sigma_P: float | None = None, V2=None, x0=None,
        tol: float = 1e-10, maxit: int = 500):
    """PCG (Sec. 3.2) on (A + diag V2 + sigma) x = b with P = (A + sigma_P)^{-1}, in the
    M-inner product <u, v>_M = sum M_idx u_idx v_idx, in which both the operator and the
    preconditioner are self-adjoint for Q^k (for k = 1, M = h I and this is textbook PCG).
    Stops when ||r||_M / ||b||_M < tol (recurrence residual).  Returns (x, iterations,
    recurrence relres, true relres)."""
    sigma_P = sigma if sigma_P is None else sigma_P
    W = mass_product(P).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    r = b - operator(P, x, sigma, V2)
    bn = np.sqrt(_mdot(W, b, b))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0, 0.0
    z = apply_inverse(P, sigma_P, r)
    p = z.copy()
    rz = _mdot(W, r, z)
    it = 0
    rel = np.sqrt(_mdot(W, r, r)) / bn
    while rel >= tol and it < maxit:
        q = operator(P, p, sigma, V2)
        alpha = rz / _mdot(W, p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = np.sqrt(_mdot(W, r, r)) / bn
        if rel < tol:
            break
        z = apply_inverse(P, sigma_P, r)
        rz_new = _mdot(W, r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    rt = b - operator(P, x, sigma, V2)
    return x, it, rel, np.sqrt(_mdot(W, rt, rt)) / bn


def ground_state_guess(P: SemPlan) -> np.ndarray:
    """Tensor product of the per-axis ground states of H_k, T_k e_1 = M_k^{-1/2} Q_k[:, 0]."""
    U = np.ones(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        U = U * P.T[a][:, 0].reshape(sh)
    return U.reshape(-1)


def inverse_iteration(P: SemPlan, shift: float, V2=None, u0=None, tol_lambda: float = 1e-12,
                      maxit: int = 200, pcg_tol: float = 1e-10, pcg_maxit: int = 500):
    """Shifted inverse iteration (Sec. 4.1) for the lowest eigenpair of A + diag V2, in the
    M-inner product: w = (A + V2 - shift)^{-1} u by PCG with P = (A - shift)^{-1},
    u = w / ||w||_M, lambda = <u, (A + V2) u>_M; stop when |d lambda| / |lambda| < tol_lambda.
    Returns (lambda, u, outer iterations, total PCG iterations)."""
    W = mass_product(P).reshape(-1)
    u = ground_state_guess(P) if u0 is None else np.asarray(u0, dtype=np.float64).reshape(-1)
    u = u / np.sqrt(_mdot(W, u, u))
    lam = _mdot(W, u, operator(P, u, 0.0, V2))
    total = 0
    for it in range(1, maxit + 1):
        w, k, _, _ = pcg(P, u, -shift, -shift, V2, None, pcg_tol, pcg_maxit)
        total += k
        u = w / np.sqrt(_mdot(W, w, w))
        lam_new = _mdot(W, u, operator(P, u, 0.0, V2))
        done = abs(lam_new - lam) < tol_lambda * abs(lam_new)
        lam = lam_new
        if done:
            return lam, u, it, total
    return lam, u, maxit, total


# -------------------------------------------------------------- multi-level transfer -----

def interpolate(Pc: SemPlan, uc, Pf: SemPlan) -> np.ndarray:
    """Tensor-product linear interpolation of the coarse grid function uc onto the fine grid
    (Sec. 5.3.1), as successive 1D piecewise-linear interpolations along each axis; the
    walls x = -L, L carry the Dirichlet zero."""
    X = np.asarray(uc, dtype=np.float64).reshape(Pc.shape())
    for a in range(Pc.d):
        xc = np.concatenate(([-Pc.L[a]], Pc.axes[a].x, [Pc.L[a]]))
        xf = Pf.axes[a].x
        ax = Pc.d - 1 - a
        Xe = np.moveaxis(X, ax, -1)
        Xe = np.concatenate((np.zeros(Xe.shape[:-1] + (1,)), Xe, np.zeros(Xe.shape[:-1] + (1,))), axis=-1)
        Y = np.apply_along_axis(lambda v: np.interp(xf, xc, v), -1, Xe)
        X = np.moveaxis(Y, -1, ax)
    return X.reshape(-1)
