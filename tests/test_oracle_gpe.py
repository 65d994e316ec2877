"""Pins of the GPE gradient-flow oracle (oracle/gpe.py) against what the paper and the
mathematics fix: the linear limit beta = 0 (the oscillator's ground state), the energy
decrease of the flow, the Euler-Lagrange equation eq. gpe at its fixed point, and the
agreement of the two flows of Sec. 4.2 on the same minimiser."""
import numpy as np
import pytest

from oracle import gpe, sem


def _grid(n=39, k=10, L=6.0, d=2):
    ax = sem.axis_1d(n, L, k)
    P0 = sem.plan((n,) * d, L, [np.zeros(n)] * d, k)
    PV = sem.plan((n,) * d, L, [ax.x ** 2] * d, k)
    V = sem.potential_sum(PV).reshape(-1)
    return P0, PV, V


def test_linear_limit_is_the_oscillator_ground_state():
    """beta = 0: the flow's fixed point is the discrete ground state of -Delta + |x|^2, whose
    eigenvalue the plan's eigendecomposition gives independently (sum of the per-axis
    lowest eigenvalues), with E = lambda / 2; both approach the closed form lambda = d = 2
    within the grid's discretisation error (Q^10 with four elements on [-6, 6]^2)."""
    P0, PV, V = _grid()
    u0 = np.ones(P0.N)
    u, E, lam, it = gpe.h1_flow(P0, V, 0.0, 20.0, 0.1, u0, maxit=2000, tol=1e-15)
    lam_min = PV.lam[0][0] + PV.lam[1][0]
    assert abs(lam - lam_min) < 1e-12 * lam_min and abs(E - 0.5 * lam_min) < 1e-12 * lam_min
    assert abs(lam - 2.0) < 1e-7
    g = sem.ground_state_guess(PV)
    g = gpe.normalize(PV, g)
    assert min(np.linalg.norm(u - g), np.linalg.norm(u + g)) < 1e-5


@pytest.mark.parametrize("beta", [10.0, 100.0])
def test_h1_flow_decreases_energy_and_solves_the_euler_lagrange_equation(beta):
    """Energy decreases monotonically (tau = 0.1, alpha = 20); at convergence
    -Delta u + V u + beta u^3 = lambda u holds (eq. gpe), lambda = (u, H_u u), and
    ||u||_L2 = 1."""
    P0, PV, V = _grid()
    u = gpe.normalize(P0, np.ones(P0.N))
    E_prev = gpe.energy(P0, V, beta, u)
    for _ in range(60):
        u = gpe.h1_flow_step(P0, V, beta, 20.0, 0.1, u)
        E = gpe.energy(P0, V, beta, u)
        assert E <= E_prev + 1e-13
        E_prev = E
    u, E, lam, it = gpe.h1_flow(P0, V, beta, 20.0, 0.1, u, maxit=5000, tol=1e-15)
    Hu = sem.operator(P0, u, 0.0, V + beta * u * u)
    assert np.sqrt(gpe.inner(P0, Hu - lam * u, Hu - lam * u)) < 1e-6 * lam
    assert abs(gpe.inner(P0, u, u) - 1.0) < 1e-13
    assert lam > E  # lambda = E + beta/4 ||u||_4^4 + ... > E for beta > 0


def test_two_flows_reach_the_same_minimiser():
    """The a_u flow (tau = 1, PCG on H_u with (-Delta + V)^{-1}) and the modified H^1 flow
    minimise the same energy on the sphere: same E, lambda and state."""
    P0, PV, V = _grid(n=29, k=10, L=5.0)
    beta = 50.0

    def residual(P, u):
        lam = gpe.eigenvalue(P, V, beta, u)
        r = sem.operator(P, u, 0.0, V + beta * u * u - sem.potential_sum(P).reshape(-1)) - lam * u
        return np.sqrt(gpe.inner(P, r, r)) / lam

    u1 = gpe.normalize(P0, np.ones(P0.N))
    for it1 in range(1, 20001):
        u1 = gpe.h1_flow_step(P0, V, beta, 20.0, 0.1, u1)
        if it1 % 20 == 0 and residual(P0, u1) < 1e-11:
            break
    u = gpe.normalize(PV, np.ones(PV.N))
    for it in range(1, 201):
        u = gpe.au_flow_step(PV, V, beta, 1.0, u)
        if residual(PV, u) < 1e-11:
            break
    E1, E = gpe.energy(P0, V, beta, u1), gpe.energy(PV, V, beta, u)
    l1, l2 = gpe.eigenvalue(P0, V, beta, u1), gpe.eigenvalue(PV, V, beta, u)
    assert abs(E - E1) < 1e-13 * E1 and abs(l2 - l1) < 1e-10 * l1
    assert np.linalg.norm(u - u1) < 1e-9 * np.linalg.norm(u1)
    assert it < it1 / 5  # the a_u metric needs far fewer steps (Sec. 4.3)


@pytest.mark.parametrize("beta", [0.0, 10.0, 100.0])
def test_energy_gradient_is_the_nonlinear_operator(beta):
    """eq. gpe is the Euler-Lagrange equation of eq. gpe_energy: the first variation of
    E(u) = 1/2 (u, (-Delta + V) u) + beta/4 (u^2, u^2) in a direction v is (H_u u, v) with
    H_u = -Delta + V + beta u^2, all inner products weighted by the quadrature masses.
    E(u + eps v) is a quartic in eps, so the central difference
    (E(u + eps v) - E(u - eps v)) / (2 eps) = (H_u u, v) + eps^2 beta (u, v^3) exactly;
    the eps^2 term is removed by taking two eps.  A wrong coefficient of the quartic term
    (beta/2 instead of beta/4), a missing 1/2 or unweighted sums all fail this."""
    P0, PV, V = _grid()
    rng = np.random.default_rng(5)
    u = gpe.normalize(P0, 1.0 + 0.3 * rng.standard_normal(P0.N))
    v = rng.standard_normal(P0.N)

    def cdiff(eps):
        return (gpe.energy(P0, V, beta, u + eps * v) - gpe.energy(P0, V, beta, u - eps * v)) / (2 * eps)

    e1, e2 = 1e-3, 5e-4
    d1, d2 = cdiff(e1), cdiff(e2)
    deriv = (d2 * e1 ** 2 - d1 * e2 ** 2) / (e1 ** 2 - e2 ** 2)  # eps^2 term eliminated
    Hu = sem.operator(P0, u, 0.0, V + beta * u * u)
    want = gpe.inner(P0, Hu, v)
    assert abs(deriv - want) < 1e-8 * abs(want)
    # the quartic term alone: (E_beta - E_0) is beta/4 (u^2, u^2), whose variation is beta (u^3, v)
    if beta > 0:
        q = lambda w: gpe.energy(P0, V, beta, w) - gpe.energy(P0, V, 0.0, w)
        cq = lambda eps: (q(u + eps * v) - q(u - eps * v)) / (2 * eps)
        dq = (cq(e2) * e1 ** 2 - cq(e1) * e2 ** 2) / (e1 ** 2 - e2 ** 2)
        want_q = beta * gpe.inner(P0, u ** 3, v)
        assert abs(dq - want_q) < 1e-8 * abs(want_q)
