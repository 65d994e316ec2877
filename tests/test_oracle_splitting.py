"""Pins of the splitting oracle (oracle/splitting.py) against what the paper and the
mathematics fix: the Gauss-Legendre rule, Yoshida's order conditions, the convergence
orders of Sec. 5.1 against a dense matrix exponential, and every error printed in Table
splitting (Q^10, 499^3, separable V1), which the separable structure reduces to 1D."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sem
from oracle import splitting as SP


@pytest.mark.parametrize("M", [1, 2, 3, 5, 7, 12])
def test_gauss_legendre_on_unit_interval(M):
    """Exact for x^p, p <= 2M - 1, on [0, 1], and for x^{2M} off by the Gauss remainder
    (M!)^4 / ((2M + 1) ((2M)!)^2); weights sum to 1; M = 1 is the midpoint and M = 2 the
    nodes 1/2 -+ 1/(2 sqrt 3)."""
    from math import factorial
    c, w = SP.gauss_legendre_01(M)
    assert abs(w.sum() - 1.0) < 1e-15
    for p in range(2 * M):
        assert abs(np.dot(w, c ** p) - 1.0 / (p + 1)) < 1e-14
    rem = factorial(M) ** 4 / ((2 * M + 1) * factorial(2 * M) ** 2)
    assert abs((1.0 / (2 * M + 1) - np.dot(w, c ** (2 * M))) - rem) < 1e-6 * rem + 2e-16
    if M == 1:
        assert c[0] == 0.5 and w[0] == 1.0
    if M == 2:
        np.testing.assert_allclose(c, [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], rtol=0, atol=1e-16)


def test_yoshida_coefficients():
    g1, g2 = SP.YOSHIDA_G1, SP.YOSHIDA_G2
    assert abs(2 * g1 + g2 - 1.0) < 1e-15
    assert abs(2 * g1 ** 3 + g2 ** 3) < 1e-14


def _dense_case():
    n, k, L = 39, 2, 4.0
    ax = sem.axis_1d(n, L, k)
    K = sem.laplacian_1d(ax)
    V = ax.x ** 2 + 3 * np.sin(ax.x) ** 2
    psi0 = np.exp(-(ax.x - 0.3) ** 2).astype(complex)
    psi0 /= np.linalg.norm(psi0)
    expA = lambda t, p: sla.expm(-1j * t * K) @ p  # noqa: E731
    expB = lambda t, p: np.exp(-1j * t * V) * p  # noqa: E731
    return K + np.diag(V), psi0, expA, expB


@pytest.mark.parametrize("method,M,lo,hi", [("qhop", 1, 1.95, 2.1), ("qhop", 3, 1.95, 2.1), ("qhop", 5, 1.95, 2.1),
                                            ("magnus2", 1, 3.8, 20), ("magnus2", 3, 3.8, 20)])
def test_convergence_orders(method, M, lo, hi):
    """Sec. 5.1: approximated qHOP is O(dt^2) for every M, approximated Magnus-2 at least
    O(dt^4) (pre-asymptotically faster for M = 3, as in the paper's own rate columns).
    1D Q^2 problem, dense e^{-iTH} as the reference."""
    H, psi0, expA, expB = _dense_case()
    T = 0.5
    ref = sla.expm(-1j * T * H) @ psi0
    e = [np.linalg.norm(SP.propagate(method, M, dt, int(round(T / dt)), psi0, expA, expB) - ref)
         for dt in (0.025, 0.0125)]
    assert lo <= np.log2(e[0] / e[1]) <= hi


def test_qhop_with_one_node_is_the_aba_midpoint_rule():
    """qHOP's product formula with M = 1 is e^{-iAh/2} e^{-iBh} e^{-iAh/2} (node h/2, weight
    1); the tables' M = 1 columns use the B-A-B Strang form instead, which differs from it
    at O(h^3) per step."""
    H, psi0, expA, expB = _dense_case()
    h = 0.01
    a = SP.qhop(h, 1, psi0, expA, expB)
    b = expA(0.5 * h, expB(h, expA(0.5 * h, psi0)))
    assert np.linalg.norm(a - b) < 1e-13
    assert np.linalg.norm(a - SP.strang(h, psi0, expA, expB)) > 1e-9


# Table splitting: dt -> errors for M = 1 (Strang), 3, 5, 7.
TABLE_SPLITTING = {
    0.1: (5.85e-1, 1.07e-1, 4.25e-2, 2.28e-2),
    0.01: (5.22e-3, 1.02e-3, 4.11e-4, 2.21e-4),
    0.005: (1.30e-3, 2.55e-4, 1.03e-4, 5.52e-5),
    0.001: (5.21e-5, 1.02e-5, 4.11e-6, 2.21e-6),
}


def test_paper_table_splitting_all_entries():
    """Table splitting: qHOP error ||psi_split(T) - psi_exact(T)||_2 at T = 0.1 for
    -Delta + V1 on [-8, 8]^3, V1 = sum_k (x_k^2 + 100 sin^2(pi x_k / 4)), Q^10 with 499^3
    DoFs, psi_0 = prod_k sin(pi (x_k + L) / 2L) normalised in l2, A = -Delta, B = V1,
    reference = the exact propagator.  Every operator is a tensor product of the same 1D
    operator, so psi_split = a x a x a and psi_exact = e x e x e with 1D vectors a, e, and
    ||a^3 - e^3||^2 = |a|^6 - 2 Re <e, a>^3 + |e|^6.  All 16 printed errors are matched to
    their three printed digits."""
    k, n, L = 10, 499, 8.0
    ax = sem.axis_1d(n, L, k)
    V1 = ax.x ** 2 + 100 * np.sin(np.pi * ax.x / 4) ** 2
    PA = sem.plan((n,), L, [np.zeros(n)], k)
    PH = sem.plan((n,), L, [V1], k)
    psi0 = np.sin(np.pi * (ax.x + L) / (2 * L)).astype(complex)
    psi0 /= np.linalg.norm(psi0)  # the 3D psi_0 = psi0 x psi0 x psi0 then has norm 1
    expA = lambda t, p: sem.apply_exp(PA, t, p)  # noqa: E731
    expB = lambda t, p: np.exp(-1j * t * V1) * p  # noqa: E731
    T = 0.1
    e = sem.apply_exp(PH, T, psi0)
    for dt, printed in TABLE_SPLITTING.items():
        for M, want in zip((1, 3, 5, 7), printed):
            a = SP.propagate("qhop", M, dt, int(round(T / dt)), psi0, expA, expB)
            err = np.sqrt(abs(np.vdot(a, a) ** 3 - 2 * np.real(np.vdot(e, a) ** 3) + np.vdot(e, e) ** 3))
            assert abs(err - want) <= 0.0051 * want, (dt, M, err, want)
