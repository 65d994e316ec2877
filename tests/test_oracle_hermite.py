"""Pins of the Hermite spectral oracle (oracle/hermite.py, Appendix app:hermite): the
Golub-Welsch nodes against numpy's Gauss-Hermite rule, exactness of D on Hermite
functions, the log-space similarity form against D^2 written out, the oscillator spectrum,
Table hermite_accuracy at n = 199 and all 16 errors of Table magnus2_hermite (separable V1,
reduced exactly to 1D)."""
import numpy as np
import pytest

from oracle import hermite as H
from oracle import splitting as SP


@pytest.mark.parametrize("n", [5, 64, 199])
def test_golub_welsch_nodes_are_the_gauss_hermite_nodes(n):
    x = H.golub_welsch_nodes(n)
    ref, _ = np.polynomial.hermite.hermgauss(n)
    assert np.max(np.abs(x - np.sort(ref))) < 1e-12


def test_diff_matrix_exact_on_hermite_functions():
    """D psi_m = psi_m' = sqrt(m/2) psi_{m-1} - sqrt((m+1)/2) psi_{m+1} at the nodes for
    m <= n - 2 (the interpolant of psi_m is psi_m itself)."""
    n = 40
    x = H.golub_welsch_nodes(n)
    D = H.diff_matrix(n)
    P = H.hermite_functions(n, x)
    for m in (0, 1, 5, 20, n - 2):
        want = (np.sqrt(m / 2) * P[m - 1] if m > 0 else 0.0) - np.sqrt((m + 1) / 2) * P[m + 1]
        assert np.max(np.abs(D @ P[m] - want)) < 1e-12


def test_log_space_form_equals_d_squared():
    """-D^2 from the skew similarity form and log weights equals D^2 written out."""
    n = 40
    D = H.diff_matrix(n)
    K0 = H.axis_1d(n).K0
    assert np.max(np.abs(K0 + D @ D)) < 1e-13 * np.max(np.abs(D @ D))


def test_oscillator_spectrum():
    """-u'' + x^2 u on R: eigenvalues 2j + 1 (the Hermite functions are its eigenfunctions)."""
    x = H.golub_welsch_nodes(64)
    P = H.plan((64,), [x ** 2])
    np.testing.assert_allclose(P.lam[0][:10], 2 * np.arange(10) + 1, rtol=0, atol=1e-11)


def test_paper_table_hermite_accuracy_n199():
    """Table hermite_accuracy, n = 199: (-Delta + V) u = f on R^3 with V of eq.
    test_potential and u* = prod_k sin(k pi (x_k + 1) / 2) / (1 + x_k^2) (k = 1, 2, 3 on
    x, y, z), f = (-Delta + V) u* from the exact second derivatives: l2 relative error
    6.31e-5 and Gauss-Hermite weighted L2 error 1.53e-5 (sum of w_i w_j w_k e^2, w the
    Gauss-Hermite weights of weight e^{-x^2}), to their printed three digits."""
    n = 199
    x = H.golub_welsch_nodes(n)
    f = [1600 * np.sin(np.pi * x / 4) ** 2 + (a + 1) * x ** 2 for a in range(3)]
    P = H.plan((n,) * 3, f)

    def factor(kk):
        s, c, g = np.sin(kk * (x + 1)), np.cos(kk * (x + 1)), 1.0 / (1.0 + x ** 2)
        u = s * g
        d2 = -kk ** 2 * s * g + 2 * kk * c * (-2 * x * g ** 2) + s * (6 * x ** 2 - 2) * g ** 3
        return u, d2

    (ux, dx), (uy, dy), (uz, dz) = factor(np.pi / 2), factor(np.pi), factor(1.5 * np.pi)
    U = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    LU = (dz[:, None, None] * uy[None, :, None] * ux[None, None, :] + uz[:, None, None] * dy[None, :, None] * ux[None, None, :]
          + uz[:, None, None] * uy[None, :, None] * dx[None, None, :])
    V = f[2][:, None, None] + f[1][None, :, None] + f[0][None, None, :]
    e = H.apply_inverse(P, 0.0, (-LU + V * U).reshape(-1)).reshape(U.shape) - U
    assert abs(np.linalg.norm(e) / np.linalg.norm(U) - 6.31e-5) < 0.006 * 6.31e-5
    _, w = np.polynomial.hermite.hermgauss(n)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    assert abs(np.sqrt(np.sum(W * e * e)) - 1.53e-5) < 0.006 * 1.53e-5


# Table magnus2_hermite: dt -> errors for Yoshida (M = 1), Magnus-2 M = 3, 5, 7.
TABLE_MAGNUS2_HERMITE = {
    0.2: (1.34e0, 1.41e0, 3.05e-1, 1.11e-1),
    0.125: (1.21e0, 4.85e-1, 3.59e-2, 8.85e-3),
    0.1: (1.52e0, 1.11e-1, 1.26e-2, 3.51e-3),
    0.05: (5.48e-1, 5.17e-3, 7.60e-4, 2.22e-4),
}


def test_paper_table_magnus2_hermite_all_entries():
    """Table magnus2_hermite: Magnus-2 via Yoshida on R^3, Hermite 499^3, complex128, T = 1,
    A = -Delta, B = V1 = sum (x_k^2 + 100 sin^2(pi x_k / 4)), psi_0 = the ground state of
    A + B (normalised in l2; reading: the only initial state that reproduces the table),
    reference = the exact propagator.  Separable, so the 3D error follows from 1D vectors
    as in Table splitting.  All 16 printed errors to their three printed digits."""
    n = 499
    x = H.golub_welsch_nodes(n)
    V1 = x ** 2 + 100 * np.sin(np.pi * x / 4) ** 2
    PA, PH = H.plan((n,), [np.zeros(n)]), H.plan((n,), [V1])
    psi0 = PH.T[0][:, 0].astype(complex)
    psi0 /= np.linalg.norm(psi0)
    expA = lambda t, p: H.apply_exp(PA, t, p)  # noqa: E731
    expB = lambda t, p: np.exp(-1j * t * V1) * p  # noqa: E731
    T = 1.0
    e = H.apply_exp(PH, T, psi0)
    for dt, printed in TABLE_MAGNUS2_HERMITE.items():
        for M, want in zip((1, 3, 5, 7), printed):
            a = SP.propagate("magnus2", M, dt, int(round(T / dt)), psi0, expA, expB)
            err = np.sqrt(abs(np.vdot(a, a) ** 3 - 2 * np.real(np.vdot(e, a) ** 3) + np.vdot(e, e) ** 3))
            assert abs(err - want) <= 0.0051 * want, (dt, M, err, want)
