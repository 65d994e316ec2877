"""CPU FP64 oracle of the Hamiltonian-simulation splittings of Sec. 5: Strang, the
approximated qHOP product formula (eq. qhop_product) and the approximated Magnus-2 by
Yoshida composition (eq. yoshida), for i d psi / dt = (A + B) psi with A applied through
an exact propagator and B a pointwise potential.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark are the only users.  The library product never imports this module, and
this module never imports the library.  Every step is applied as the paper writes it,
factor by factor, without merging adjacent propagations (merging is the library's
optimisation; the comparison checks it).

Operators are passed as callables: expA(tau, psi) = e^{-i tau A} psi and
expB(theta, psi) = e^{-i theta B} psi (any tau, theta, negative ones included).
"""
from __future__ import annotations

import numpy as np

# Yoshida's fourth-order composition coefficients (eq. yoshida): 2 g1 + g2 = 1 and
# 2 g1^3 + g2^3 = 0.
YOSHIDA_G1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
YOSHIDA_G2 = -(2.0 ** (1.0 / 3.0)) / (2.0 - 2.0 ** (1.0 / 3.0))


def gauss_legendre_01(M: int):
    """Gauss-Legendre nodes c_k in (0, 1), ascending, and weights w_k with sum 1 (the
    normalised weights of Sec. 5.1): the M-point rule on [-1, 1] mapped onto [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(M)
    return 0.5 * (x + 1.0), 0.5 * w


def strang(h, psi, expA, expB):
    """e^{-i B h/2} e^{-i A h} e^{-i B h/2} psi: the Strang step of the tables' M = 1
    columns (one A-propagation, Remark cost_naive_merged)."""
    psi = expB(0.5 * h, psi)
    psi = expA(h, psi)
    return expB(0.5 * h, psi)


def qhop(h, M, psi, expA, expB):
    """One approximated qHOP step P(h) = e^{-iAh} prod_{k=1..M} e^{-i w_k h H_I(s_k)},
    s_k = c_k h, with each factor e^{-i w h H_I(s)} = e^{iAs} e^{-i w h B} e^{-iAs} applied
    exactly; factor k = 1 acts first (eq. qhop_product and the merged form of Remark
    cost_naive_merged).  (2M + 1) A-propagations as written."""
    c, w = gauss_legendre_01(M)
    for k in range(M):
        s = c[k] * h
        psi = expA(s, psi)            # e^{-iA s_k}
        psi = expB(w[k] * h, psi)     # e^{-i w_k h B}
        psi = expA(-s, psi)           # e^{+iA s_k}
    return expA(h, psi)


def step(method: str, M: int, h, psi, expA, expB):
    """One time step of size h.  method "qhop": the qHOP step for M >= 2, Strang for M = 1
    (the tables' M = 1 column); "magnus2": the Yoshida composition
    P(g1 h) P(g2 h) P(g1 h) of that step (eq. yoshida; M = 1 is plain Yoshida)."""
    one = (lambda hh, p: strang(hh, p, expA, expB)) if M == 1 else (lambda hh, p: qhop(hh, M, p, expA, expB))
    if method == "qhop":
        return one(h, psi)
    if method == "magnus2":
        psi = one(YOSHIDA_G1 * h, psi)
        psi = one(YOSHIDA_G2 * h, psi)
        return one(YOSHIDA_G1 * h, psi)
    raise ValueError(method)


def propagate(method: str, M: int, dt, nsteps: int, psi, expA, expB):
    for _ in range(nsteps):
        psi = step(method, M, dt, psi, expA, expB)
    return psi
