"""CPU FP64 oracle of the Gross-Pitaevskii ground state by Riemannian (Sobolev) gradient
flows on the L2 unit sphere (Sec. 4.2-4.3): the modified H^1 flow and the a_u flow, on a
Q^k spectral element plan (oracle/sem.py).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark are the only users.  The library product never imports this module, and
this module never imports the library.

Discrete setting (GLL quadrature, M = the lumped mass):
    (u, v) = sum_idx M_idx u_idx v_idx,   ||u||_L2^2 = (u, u),
    H_u = -Delta + V + beta u^2   (K_k = M_k^{-1} Stiff_k on every axis),
    E(u) = 1/2 (u, (-Delta + V) u) + beta/4 (u^2, u^2)          (eq. gpe_energy),
    lambda(u) = (u, H_u u).
One step of either flow (eq. riemannian_update):
    u <- (u - tau grad) / ||u - tau grad||,
    grad = G H_u u - [(u, G H_u u) / (u, G u)] G u,
the Riemannian gradient of E in the metric g whose Riesz map is G^{-1}: the g-gradient of E
projected g-orthogonally onto the tangent space {w : (w, u) = 0} of the sphere.
    modified H^1 (eq. h1_metric):  G = (-Delta + alpha)^{-1}        (two direct solves);
    a_u (eq. au_metric):           G = (-Delta + V + beta u^2)^{-1}  (PCG with the
                                   preconditioner (-Delta + V)^{-1}).
"""
from __future__ import annotations

import numpy as np

from oracle import sem


def inner(P, u, v) -> float:
    return float(np.sum(sem.mass_product(P).reshape(-1) * u * v))


def normalize(P, u):
    return u / np.sqrt(inner(P, u, u))


def energy(P, V, beta, u) -> float:
    """E(u) of eq. gpe_energy with GLL quadrature; V: the potential at the nodes (N)."""
    Hu = sem.operator(P, u, 0.0, V - sem.potential_sum(P).reshape(-1))
    return 0.5 * inner(P, u, Hu) + 0.25 * beta * inner(P, u * u, u * u)


def eigenvalue(P, V, beta, u) -> float:
    """lambda(u) = (u, (-Delta + V + beta u^2) u)."""
    Hu = sem.operator(P, u, 0.0, V + beta * u * u - sem.potential_sum(P).reshape(-1))
    return inner(P, u, Hu)


def h1_flow_step(P0, V, beta, alpha, tau, u):
    """One modified H^1 step; P0 is the plan of -Delta alone (f = 0) and G = (-Delta + alpha)^{-1}
    its direct inverse with sigma = alpha."""
    r = sem.operator(P0, u, 0.0, V + beta * u * u)    # H_u u
    w1 = sem.apply_inverse(P0, alpha, r)               # G H_u u
    w2 = sem.apply_inverse(P0, alpha, u)               # G u
    grad = w1 - (inner(P0, u, w1) / inner(P0, u, w2)) * w2
    return normalize(P0, u - tau * grad)


def au_flow_step(PV, V1, beta, tau, u, pcg_tol=1e-13):
    """One a_u step; PV is the plan of -Delta + V1 (V = V1 separable here), G H_u u and G u
    solved by PCG on -Delta + V1 + beta u^2 with the preconditioner (-Delta + V1)^{-1}.
    G H_u u = u exactly, so only G u needs a solve (the second solve of the paper's count
    is this identity)."""
    V2 = beta * u * u
    w2, _, _, _ = sem.pcg(PV, u, 0.0, 0.0, V2, tol=pcg_tol, maxit=2000)
    grad = u - (inner(PV, u, u) / inner(PV, u, w2)) * w2
    return normalize(PV, u - tau * grad)


def h1_flow(P0, V, beta, alpha, tau, u0, maxit=5000, tol=1e-14, E_ref=None):
    """Runs the modified H^1 flow from u0 until |E_k - E_{k-1}| / |E_k| < tol (or, when E_ref
    is given, |E_k - E_ref| / |E_ref| < tol).  Returns (u, E, lambda, iterations)."""
    u = normalize(P0, np.asarray(u0, dtype=np.float64))
    E = energy(P0, V, beta, u)
    for it in range(1, maxit + 1):
        u = h1_flow_step(P0, V, beta, alpha, tau, u)
        E_new = energy(P0, V, beta, u)
        done = abs(E_new - (E if E_ref is None else E_ref)) < tol * abs(E_new)
        E = E_new
        if done:
            return u, E, eigenvalue(P0, V, beta, u), it
    return u, E, eigenvalue(P0, V, beta, u), maxit
