"""Pins of the Q^k spectral element oracle (oracle/sem.py) against what the paper and the
mathematics fix, independently of the oracle's own formulas: textbook GLL rules, exact
polynomial integrals, the finite-difference special case k = 1, closed-form spectra, the
eigenvalues the paper prints (Tables inverse_iter and multilevel), the convergence order
it states for Q^k (Sec. 2), and dense brute force on small grids."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import Polynomial

import oracle
from oracle import sem


# ------------------------------------------------------------------- GLL rule ------------

@pytest.mark.parametrize("k,nodes,weights", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_gll_closed_forms(k, nodes, weights):
    """Textbook Gauss-Lobatto-Legendre points and weights (Abramowitz & Stegun 25.4.32)."""
    xi, w = sem.gll(k)
    np.testing.assert_allclose(xi, nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, weights, rtol=1e-14)


@pytest.mark.parametrize("k", [2, 3, 5, 8, 10, 16, 20])
def test_gll_quadrature_degree(k):
    """The (k+1)-point GLL rule integrates x^p exactly for p <= 2k - 1; for p = 2k its error is
    the Lobatto remainder (Abramowitz & Stegun 25.4.32) with f^(2m-2) = (2m-2)!, m = k + 1:
    int - sum = -m (m-1)^3 2^(2m-1) ((m-2)!)^4 / ((2m-1) ((2m-2)!)^2)."""
    from math import factorial
    xi, w = sem.gll(k)
    for p in range(2 * k):
        exact = 2.0 / (p + 1) if p % 2 == 0 else 0.0
        assert abs(np.dot(w, xi ** p) - exact) < 1e-13, p
    m = k + 1
    rem = -m * (m - 1) ** 3 * 2.0 ** (2 * m - 1) * factorial(m - 2) ** 4 / ((2 * m - 1) * factorial(2 * m - 2) ** 2)
    err = 2.0 / (2 * k + 1) - np.dot(w, xi ** (2 * k))
    assert abs(err - rem) < 1e-6 * abs(rem) + 1e-14


@pytest.mark.parametrize("k", [2, 4, 7, 10, 20])
def test_diff_matrix_exact_on_polynomials(k):
    """D maps nodal values of any polynomial of degree <= k to the nodal values of its
    derivative."""
    xi, _ = sem.gll(k)
    D = sem.diff_matrix(xi)
    rng = np.random.default_rng(k)
    for _ in range(3):
        p = Polynomial(rng.standard_normal(k + 1))
        np.testing.assert_allclose(D @ p(xi), p.deriv()(xi), rtol=0, atol=1e-10 * (1 + k * k))


@pytest.mark.parametrize("k", [1, 2, 3, 6, 10])
def test_element_stiffness_is_the_exact_galerkin_integral(k):
    """For polynomials p, q of degree <= k on one element [a, a + h], the GLL stiffness gives
    p^T Se q = int_a^{a+h} p'(x) q'(x) dx exactly (the integrand has degree 2k - 2); the
    lumped mass sums to h."""
    a, h = -0.3, 0.7
    Se, me = sem.element_matrices(k, h)
    xi, _ = sem.gll(k)
    x = a + 0.5 * (xi + 1.0) * h
    rng = np.random.default_rng(10 + k)
    for _ in range(3):
        p = Polynomial(rng.standard_normal(k + 1))
        q = Polynomial(rng.standard_normal(k + 1))
        prim = (p.deriv() * q.deriv()).integ()
        exact = prim(a + h) - prim(a)
        assert abs(p(x) @ Se @ q(x) - exact) < 1e-11 * (1 + abs(exact))
    assert abs(me.sum() - h) < 1e-15
    np.testing.assert_allclose(Se @ np.ones(k + 1), 0.0, atol=1e-11)  # constants have no energy


def test_q1_is_the_second_order_finite_difference_scheme():
    """k = 1: uniform interior nodes x_i = -L + i h, M = h I, K = h^-2 tridiag(-1, 2, -1) --
    the operator of the Q^1 oracle (oracle.c), itself pinned to the dense Kronecker sum."""
    n, L = 37, 3.5
    ax = sem.axis_1d(n, L, 1)
    np.testing.assert_allclose(ax.x, oracle.grid(n, L), rtol=0, atol=1e-14)
    h = 2 * L / (n + 1)
    np.testing.assert_allclose(ax.m, h, rtol=1e-15)
    np.testing.assert_allclose(sem.laplacian_1d(ax), oracle.operator_1d(n, L, np.zeros(n)), rtol=1e-13, atol=1e-12)


def test_elements_tile_the_interval():
    """Nodes are strictly increasing inside (-L, L), with c - 1 element end points at
    -L + e h_e, and the lumped masses add up to the length 2L minus the two boundary masses."""
    k, c, L = 5, 7, 2.0
    n = c * k - 1
    ax = sem.axis_1d(n, L, k)
    assert np.all(np.diff(ax.x) > 0) and ax.x[0] > -L and ax.x[-1] < L
    he = 2 * L / c
    np.testing.assert_allclose(ax.x[k - 1::k][:c - 1], -L + he * np.arange(1, c), rtol=0, atol=1e-14)
    _, w = sem.gll(k)
    np.testing.assert_allclose(ax.m.sum(), 2 * L - he * w[0], rtol=1e-14)


# ------------------------------------------------------------- spectra and the paper ----

@pytest.mark.parametrize("gamma", [1.0, 2.0])
def test_harmonic_oscillator_spectrum(gamma):
    """-u'' + gamma^2 x^2 u on [-8, 8] (the Gaussian tails are below 1e-20 at the walls):
    eigenvalues gamma (2j + 1).  Q^10 with 16 elements reaches them to rounding."""
    k, c, L = 10, 16, 8.0
    n = c * k - 1
    ax = sem.axis_1d(n, L, k)
    P = sem.plan((n,), L, [gamma ** 2 * ax.x ** 2], k)
    np.testing.assert_allclose(P.lam[0][:5], gamma * (2 * np.arange(5) + 1), rtol=5e-12, atol=0)


def test_paper_ground_state_eigenvalue_q10():
    """Table inverse_iter: -Delta + V1 on [-8, 8]^3 with V1 = sum_k (x_k^2 + 100 sin^2(pi x_k / 4)),
    Q^10, lambda_1 = 23.2878438176.  V1 is separable with the same term on each axis, so
    lambda_1 is 3 times the lowest eigenvalue of the 1D operator; at n = 599 (the table's
    599^3 grid) it agrees to within half a unit of the last printed digit."""
    k, n, L = 10, 599, 8.0
    ax = sem.axis_1d(n, L, k)
    P = sem.plan((n,), L, [ax.x ** 2 + 100 * np.sin(np.pi * ax.x / 4) ** 2], k)
    assert abs(3 * P.lam[0][0] - 23.2878438176) < 5e-11


def test_paper_ground_state_eigenvalue_stirrer_q20():
    """Table multilevel: H = -Delta + x^2 + y^2 + 4 z^2 + 8 exp(-((x - 1)^2 + y^2)) on [-8, 8]^3
    (eq. stirrer with gamma = (1, 1, 2), w_0 = 4, delta = 1, r_0 = 1), Q^20,
    lambda_1 = 5.286155366963.  V2 does not depend on z, so H = H_xy + H_z and lambda_1 is the
    lowest eigenvalue of the 2D operator in (x, y) plus that of -d^2/dz^2 + 4 z^2 (= 2, the
    oscillator's ground state).  The 2D problem is solved in its symmetric form
    M^{-1/2} Stiff M^{-1/2} with a sparse shift-invert Lanczos; n = 99 per axis."""
    k, n, L = 20, 99, 8.0
    ax = sem.axis_1d(n, L, k)
    r = 1.0 / np.sqrt(ax.m)
    Ks = sp.csr_matrix(r[:, None] * ax.stiff * r[None, :])
    I = sp.identity(n, format="csr")
    X, Y = np.meshgrid(ax.x, ax.x, indexing="xy")
    V = X ** 2 + Y ** 2 + 8.0 * np.exp(-((X - 1.0) ** 2 + Y ** 2))
    A = (sp.kron(I, Ks) + sp.kron(Ks, I) + sp.diags(V.reshape(-1))).tocsc()
    mu_xy = spla.eigsh(A, k=1, sigma=3.0, which="LM", return_eigenvectors=False)[0]
    Pz = sem.plan((n,), L, [4.0 * ax.x ** 2], k)
    assert abs(Pz.lam[0][0] - 2.0) < 1e-12
    assert abs(mu_xy + Pz.lam[0][0] - 5.286155366963) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_convergence_order(k):
    """Sec. 2: Q^k SEM is a (k + 2)-th order scheme in the l2 norm over node values for
    k >= 2 (second order for k = 1).  1D problem of the paper's 3D test (eq. test_potential,
    x-term): -u'' + (1600 sin^2(pi x / 4) + x^2) u = f on [-1, 1], u* = sin(pi x)."""
    def err(c):
        n = c * k - 1
        ax = sem.axis_1d(n, 1.0, k)
        V = 1600 * np.sin(np.pi * ax.x / 4) ** 2 + ax.x ** 2
        us = np.sin(np.pi * ax.x)
        P = sem.plan((n,), 1.0, [V], k)
        u = sem.apply_inverse(P, 0.0, np.pi ** 2 * us + V * us)
        return np.linalg.norm(u - us) / np.linalg.norm(us)
    order = np.log2(err(20) / err(40))
    expect = 2 if k == 1 else k + 2
    assert abs(order - expect) < 0.15, order


# ------------------------------------------------------------- 4-step vs dense -----------

CASES = [((8, 11), 3, (1.5, 2.0)), ((5, 7, 3), 2, (1.0, 1.5, 0.8)), ((9, 9), 5, (2.0, 2.0)), ((6, 4, 5), 1, (1.0, 1.0, 1.0))]


def _case(n, k, L, seed=0):
    rng = np.random.default_rng(seed)
    f = []
    for a in range(len(n)):
        x = sem.axis_1d(n[a], L[a], k).x
        f.append(0.7 * x ** 2 + 0.3 * np.sin(x) ** 2)
    P = sem.plan(n, L, f, k)
    return P, rng


@pytest.mark.parametrize("n,k,L", CASES)
def test_apply_inverse_equals_dense_solve(n, k, L):
    P, rng = _case(n, k, L)
    b = rng.standard_normal(P.N)
    A = sem.dense_operator(P, 0.8)
    u = sem.apply_inverse(P, 0.8, b)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("n,k,L", CASES)
def test_apply_exp_equals_dense_expm(n, k, L):
    P, rng = _case(n, k, L, 1)
    psi = rng.standard_normal(P.N) + 1j * rng.standard_normal(P.N)
    A = sem.dense_operator(P)
    ref = sla.expm(-1j * 0.01 * A) @ psi
    out = sem.apply_exp(P, 0.01, psi)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-11


@pytest.mark.parametrize("n,k,L", CASES)
def test_operator_is_the_dense_matrix_and_m_self_adjoint(n, k, L):
    P, rng = _case(n, k, L, 2)
    V2 = rng.uniform(0, 2, P.N)
    x, y = rng.standard_normal(P.N), rng.standard_normal(P.N)
    A = sem.dense_operator(P, 0.3, V2)
    np.testing.assert_allclose(sem.operator(P, x, 0.3, V2), A @ x, rtol=1e-13, atol=1e-10)
    W = sem.mass_product(P).reshape(-1)
    lhs = np.sum(W * x * sem.operator(P, y, 0.3, V2))
    rhs = np.sum(W * sem.operator(P, x, 0.3, V2) * y)
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1)


@pytest.mark.parametrize("n,k,L", CASES)
def test_pcg_and_inverse_iteration_equal_dense(n, k, L):
    P, rng = _case(n, k, L, 3)
    V2 = rng.uniform(0, 3, P.N)
    b = rng.standard_normal(P.N)
    A = sem.dense_operator(P, 0.5, V2)
    x, it, rel, true_rel = sem.pcg(P, b, 0.5, 0.5, V2, tol=1e-12)
    ref = np.linalg.solve(A, b)
    assert it > 1 and rel < 1e-12 and true_rel < 1e-11
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10
    ev = np.sort(np.real(np.linalg.eigvals(sem.dense_operator(P, 0.0, V2))))
    shift = ev[0] - 1.0
    lam, u, outer, _ = sem.inverse_iteration(P, shift, V2, tol_lambda=1e-13, pcg_tol=1e-12)
    assert abs(lam - ev[0]) < 1e-10 * abs(ev[0])
    Hu = sem.operator(P, u, 0.0, V2)
    assert np.linalg.norm(Hu - lam * u) < 1e-6 * np.linalg.norm(Hu)


def test_interpolation_identity_and_multilinear_exactness():
    """Tensor-product linear interpolation is the identity onto the same grid, and exact
    for functions linear in each variable at fine nodes between interior coarse nodes."""
    Pc = sem.plan((9, 14), (2.0, 3.0), [np.zeros(9), np.zeros(14)], 5)
    Pf = sem.plan((39, 23), (2.0, 3.0), [np.zeros(39), np.zeros(23)], 2)
    xc, yc = Pc.axes[0].x, Pc.axes[1].x
    Uc = (1.0 + 0.3 * xc[None, :]) * (2.0 - 0.7 * yc[:, None])
    np.testing.assert_allclose(sem.interpolate(Pc, Uc.reshape(-1), Pc), Uc.reshape(-1), rtol=0, atol=1e-15)
    Uf = sem.interpolate(Pc, Uc.reshape(-1), Pf).reshape(23, 39)
    xf, yf = Pf.axes[0].x, Pf.axes[1].x
    ix = (xf >= xc[0]) & (xf <= xc[-1])
    iy = (yf >= yc[0]) & (yf <= yc[-1])
    want = (1.0 + 0.3 * xf[None, :]) * (2.0 - 0.7 * yf[:, None])
    np.testing.assert_allclose(Uf[np.ix_(iy, ix)], want[np.ix_(iy, ix)], rtol=1e-14, atol=1e-14)
    # beyond the outermost coarse nodes the interpolant falls linearly to the wall's zero
    j = np.argmax(~ix)
    assert abs(Uf[np.argmax(iy), j]) < abs(want[np.argmax(iy), j])
