"""The host tridiagonal eigensolver of plan creation (ts_tridiag_eig, step 1 of Sec. 2.1 for
the Q^1 operator): implicit symmetric QR with the Wilkinson shift.  Checked without a GPU
against the closed-form Dirichlet finite-difference spectrum, LAPACK on random matrices,
the oracle's Jacobi decomposition of the harmonic Q^1 operator, and hard cases (an already
diagonal matrix, exactly repeated eigenvalues, the nearly degenerate pairs of Wilkinson's
W21+)."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def T():
    from paper_2605_20491_b300 import build, tschrod
    build.build()
    return tschrod


def check_decomposition(lam, Z, a, b, tol=4e-15):
    n = a.size
    Tm = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    scale = max(np.abs(a).max() + 2 * (np.abs(b).max() if b.size else 0.0), 1e-300)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(Z.T @ Z - np.eye(n)).max() < tol * n
    assert np.abs(Tm @ Z - Z * lam[None, :]).max() < tol * n * scale


@pytest.mark.parametrize("n", [1, 2, 3, 31, 128, 192])
def test_dirichlet_closed_form(T, n):
    """h^-2 tridiag(-1, 2, -1): lambda_j = 4 h^-2 sin^2(j pi / (2 (n + 1))), eigenvectors
    sin(i j pi / (n + 1)) normalised."""
    h = 16.0 / (n + 1)
    a, b = np.full(n, 2 / h ** 2), np.full(n - 1, -1 / h ** 2)
    lam, Z = T.ts_tridiag_eig(a, b)
    j = np.arange(1, n + 1)
    exact = 4 / h ** 2 * np.sin(j * np.pi / (2 * (n + 1))) ** 2
    assert np.abs(lam - exact).max() < 4e-15 * n * exact.max()
    V = np.sin(np.outer(j, j) * np.pi / (n + 1))
    V /= np.linalg.norm(V, axis=0)
    assert np.abs(np.abs(np.sum(V * Z, axis=0)) - 1).max() < 1e-12
    check_decomposition(lam, Z, a, b)


@pytest.mark.parametrize("seed,n", [(0, 5), (1, 64), (2, 97), (3, 160)])
def test_random_against_lapack(T, seed, n):
    rng = np.random.default_rng(seed)
    a, b = rng.standard_normal(n) * 10, rng.standard_normal(n - 1)
    lam, Z = T.ts_tridiag_eig(a, b)
    ref = np.linalg.eigvalsh(np.diag(a) + np.diag(b, 1) + np.diag(b, -1))
    assert np.abs(lam - ref).max() < 1e-14 * n * np.abs(ref).max()
    check_decomposition(lam, Z, a, b)


def test_harmonic_q1_operator_against_oracle(T):
    """The Q^1 operator of a plan axis (n = 70 on [-8, 8], f = (1.3 x)^2): the oracle's
    Jacobi eigenvalues."""
    n, L = 70, 8.0
    h = 2 * L / (n + 1)
    x = -L + h * np.arange(1, n + 1)
    f = (1.3 * x) ** 2
    Po = O.plan((n,), (L,), [f])
    lam, Z = T.ts_tridiag_eig(2 / h ** 2 + f, np.full(n - 1, -1 / h ** 2))
    assert np.abs(lam - Po.lam[0]).max() < 1e-13 * np.abs(Po.lam[0]).max()
    check_decomposition(lam, Z, 2 / h ** 2 + f, np.full(n - 1, -1 / h ** 2))


def test_hard_cases(T):
    # already diagonal, unsorted
    a = np.array([3.0, -1.0, 2.0, 2.0, 0.0])
    lam, Z = T.ts_tridiag_eig(a, np.zeros(4))
    assert np.array_equal(lam, np.sort(a))
    check_decomposition(lam, Z, a, np.zeros(4))
    # two identical blocks, decoupled: every eigenvalue exactly twice
    blk_a, blk_b = np.array([2.0, 1.0, 3.0]), np.array([0.5, -0.7])
    a = np.concatenate([blk_a, blk_a])
    b = np.concatenate([blk_b, [0.0], blk_b])
    lam, Z = T.ts_tridiag_eig(a, b)
    assert np.abs(lam[0::2] - lam[1::2]).max() < 1e-15 * 4
    check_decomposition(lam, Z, a, b)
    # Wilkinson W21+: pairs that agree to ~1e-13 and beyond
    a = np.abs(np.arange(-10, 11)).astype(float)
    b = np.ones(20)
    lam, Z = T.ts_tridiag_eig(a, b)
    assert lam[-1] - lam[-2] < 1e-12
    check_decomposition(lam, Z, a, b)
    # n = 1
    lam, Z = T.ts_tridiag_eig(np.array([4.5]), np.zeros(0))
    assert lam[0] == 4.5 and Z[0, 0] == 1.0


def test_invalid_arguments(T):
    with pytest.raises(T.TsError) as e:
        T.ts_tridiag_eig(np.array([1.0, np.nan]), np.array([1.0]))
    assert e.value.status == T.TS_ERR_INVALID_ARG
    with pytest.raises(T.TsError) as e:
        T.ts_tridiag_eig(np.zeros(0), np.zeros(0))
    assert e.value.status == T.TS_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [16, 17, 64, 97, 128, 191])
def test_persymmetric_split(T, n):
    """A matrix symmetric about its middle (a potential symmetric on a symmetric grid) is
    solved as two half-size problems of even and odd eigenvectors: the same spectrum as
    LAPACK, orthonormal eigenvectors of the right parity, for even and odd n, random
    entries and a double-well potential whose lowest pairs are nearly degenerate."""
    rng = np.random.default_rng(n)
    half_a, half_b = rng.standard_normal((n + 1) // 2) * 5, rng.standard_normal(n // 2)
    a = np.concatenate([half_a, half_a[: n // 2][::-1]])
    b = np.concatenate([half_b, half_b[: (n - 1) // 2][::-1]])
    h = 10.0 / (n + 1)
    x = -5.0 + h * np.arange(1, n + 1)
    well_a = 2 / h ** 2 + 4.0 * (x ** 2 - 4.0) ** 2
    for aa, bb in ((a, b), (well_a, np.full(n - 1, -1 / h ** 2))):
        lam, Z = T.ts_tridiag_eig(aa, bb)
        ref = np.linalg.eigvalsh(np.diag(aa) + np.diag(bb, 1) + np.diag(bb, -1))
        assert np.abs(lam - ref).max() < 1e-14 * n * np.abs(ref).max()
        check_decomposition(lam, Z, aa, bb)
        parity = np.sum(Z * Z[::-1, :], axis=0)  # +1 even, -1 odd
        assert np.abs(np.abs(parity) - 1).max() < 1e-12


def test_nearly_persymmetric_inputs(T):
    """Entries symmetric only to rounding (a grid computed in floating point) take the split
    with the mirrored pairs averaged: the decomposition still satisfies the input to
    rounding.  An asymmetry well above rounding takes the plain QR."""
    n = 80
    h = 16.0 / (n + 1)
    x = -8.0 + h * np.arange(1, n + 1)
    a = 2 / h ** 2 + (1.3 * x) ** 2
    b = np.full(n - 1, -1 / h ** 2)
    assert not np.array_equal(a, a[::-1])  # the float grid is not exactly symmetric
    lam, Z = T.ts_tridiag_eig(a, b)
    check_decomposition(lam, Z, a, b)
    skew = a + 1e-6 * x  # an odd term: no symmetry
    lam2, Z2 = T.ts_tridiag_eig(skew, b)
    ref = np.linalg.eigvalsh(np.diag(skew) + np.diag(b, 1) + np.diag(b, -1))
    assert np.abs(lam2 - ref).max() < 1e-14 * n * np.abs(ref).max()
    check_decomposition(lam2, Z2, skew, b)
