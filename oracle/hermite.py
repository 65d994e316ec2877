"""CPU FP64 oracle of the Hermite spectral discretisation on R^d (Appendix app:hermite) and
the tensor-product solver on it.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark are the only users.  The library product never imports this module, and
this module never imports the library.

Per axis, with n nodes:
* the nodes x_j are the eigenvalues of the symmetric tridiagonal J with J_{k,k} = 0 and
  J_{k,k+1} = J_{k+1,k} = sqrt(k/2) (Golub-Welsch), i.e. the roots of H_n;
* psi_m are the normalised Hermite functions, by the recurrence
  psi_0 = pi^{-1/4} e^{-x^2/2}, psi_{m+1} = sqrt(2/(m+1)) x psi_m - sqrt(m/(m+1)) psi_{m-1};
* D_ij = psi_{n-1}(x_i) / (psi_{n-1}(x_j) (x_i - x_j)) for i != j, D_ii = 0;
* K = -D^2 + diag f(x_j), eigendecomposed as K = T Lambda T^{-1}.
D is similar to the skew matrix B_ij = s_i s_j / (x_i - x_j) (s = sign psi_{n-1}(x_j)) by the
diagonal W^{1/2}, W_j = 1 / (n psi_{n-1}(x_j)^2) (the Gauss weights of Hermite functions):
-D^2 + F = W^{-1/2} (-B^2 + F) W^{1/2}, so K is diagonalised through the symmetric
-B^2 + F = Q Lambda Q^T with T = W^{-1/2} Q, T^{-1} = Q^T W^{1/2}.  psi_{n-1} is evaluated in
log form (the plain recurrence underflows with e^{-x^2/2} from n ~ 745); W itself stays
moderate, since every node lies where psi_{n-1} oscillates.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from oracle import sem


def golub_welsch_nodes(n: int) -> np.ndarray:
    k = np.arange(1, n)
    J = np.diag(np.sqrt(k / 2.0), 1) + np.diag(np.sqrt(k / 2.0), -1)
    return np.linalg.eigvalsh(J)


def hermite_functions(m_max: int, x):
    """psi_0 .. psi_{m_max} at x (rows), by the three-term recurrence (fine while the
    values stay above the FP64 underflow threshold)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((m_max + 1,) + x.shape)
    out[0] = np.pi ** -0.25 * np.exp(-0.5 * x * x)
    if m_max >= 1:
        out[1] = np.sqrt(2.0) * x * out[0]
    for m in range(1, m_max):
        out[m + 1] = np.sqrt(2.0 / (m + 1)) * x * out[m] - np.sqrt(m / (m + 1.0)) * out[m - 1]
    return out


def log_abs_psi_last(n: int, x):
    """log |psi_{n-1}(x)| and its sign, by the recurrence on the polynomial part
    (psi_m = p_m e^{-x^2/2}) with periodic rescaling, so that nothing under- or overflows."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.full_like(x, np.pi ** -0.25)
    logs = np.zeros_like(x)
    if n == 1:
        return np.log(np.abs(p0)) - 0.5 * x * x, np.sign(p0)
    p1 = np.sqrt(2.0) * x * p0
    for m in range(1, n - 1):
        p2 = np.sqrt(2.0 / (m + 1)) * x * p1 - np.sqrt(m / (m + 1.0)) * p0
        p0, p1 = p1, p2
        big = np.abs(p1) > 1e100
        if np.any(big):
            p0 = np.where(big, p0 * 1e-100, p0)
            p1 = np.where(big, p1 * 1e-100, p1)
            logs = logs + np.where(big, np.log(1e100), 0.0)
    return np.log(np.abs(p1)) + logs - 0.5 * x * x, np.sign(p1)


@dataclass
class HermiteAxis:
    x: np.ndarray
    log_w: np.ndarray   # log of W_j = 1 / (n psi_{n-1}(x_j)^2)
    B: np.ndarray       # the skew-symmetric similarity form of D
    K0: np.ndarray      # -D^2 (user frame), from -B^2 and the weights


def axis_1d(n: int) -> HermiteAxis:
    x = golub_welsch_nodes(n)
    lp, sg = log_abs_psi_last(n, x)
    log_w = -np.log(n) - 2.0 * lp
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    B = (sg[:, None] * sg[None, :]) / diff
    np.fill_diagonal(B, 0.0)
    # -D^2 = W^{-1/2} (-B^2) W^{1/2}:  (K0)_ij = exp((log_w_j - log_w_i) / 2) (-B^2)_ij
    K0 = np.exp(0.5 * (log_w[None, :] - log_w[:, None])) * (-(B @ B))
    return HermiteAxis(x, log_w, B, K0)


def diff_matrix(n: int) -> np.ndarray:
    """D exactly as the appendix writes it (for moderate n, where psi_{n-1} does not underflow)."""
    x = golub_welsch_nodes(n)
    psi = hermite_functions(n - 1, x)[n - 1]
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    D = psi[:, None] / (psi[None, :] * diff)
    np.fill_diagonal(D, 0.0)
    return D


@dataclass
class HermitePlan:
    n: tuple
    axes: list = field(default_factory=list)
    f: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    T: list = field(default_factory=list)
    Tinv: list = field(default_factory=list)

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def shape(self):
        return tuple(reversed(self.n))


def plan(n, f) -> HermitePlan:
    """Per axis: -B^2 + diag f = Q Lambda Q^T (symmetric), T = W^{-1/2} Q, T^{-1} = Q^T W^{1/2}."""
    P = HermitePlan(tuple(int(v) for v in n))
    for a, na in enumerate(P.n):
        ax = axis_1d(na)
        fa = np.asarray(f[a], dtype=np.float64)
        Hs = -(ax.B @ ax.B) + np.diag(fa)
        lam, Q = np.linalg.eigh(0.5 * (Hs + Hs.T))
        P.axes.append(ax)
        P.f.append(fa)
        P.lam.append(lam)
        P.T.append(np.exp(-0.5 * ax.log_w)[:, None] * Q)
        P.Tinv.append(Q.T * np.exp(0.5 * ax.log_w)[None, :])
    return P


def apply_inverse(P: HermitePlan, sigma: float, b) -> np.ndarray:
    X = np.asarray(b, dtype=np.float64).reshape(P.shape())
    for a in range(P.d):
        X = sem.along(P, a, P.Tinv[a], X)
    S = np.zeros(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        S = S + P.lam[a].reshape(sh)
    X = X / (S + sigma)
    for a in range(P.d):
        X = sem.along(P, a, P.T[a], X)
    return X.reshape(-1)


def apply_exp(P: HermitePlan, tau: float, psi) -> np.ndarray:
    X = np.asarray(psi, dtype=np.complex128).reshape(P.shape())
    for a in range(P.d):
        X = sem.along(P, a, P.Tinv[a], X)
    S = np.zeros(P.shape())
    for a in range(P.d):
        sh = [1] * P.d
        sh[P.d - 1 - a] = P.n[a]
        S = S + P.lam[a].reshape(sh)
    X = X * np.exp(-1j * tau * S)
    for a in range(P.d):
        X = sem.along(P, a, P.T[a], X)
    return X.reshape(-1)
