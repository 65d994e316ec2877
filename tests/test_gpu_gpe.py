"""GPE ground state (Sec. 4.2-4.3) on the GPU through ts_gpe_ground_state: element-wise
parity with the oracle's gradient flows (oracle/gpe.py) over a fixed number of steps, and
the energies and eigenvalues of Table h1_flow (beta = 10, 100, eigenfunction initial
guess, Q^20 on [-8, 8]^3)."""
import numpy as np
import pytest

from oracle import gpe, sem
from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def _case(T, n, k, L, mask=0):
    f = [0.8 * sem.axis_1d(n[a], L[a], k).x ** 2 for a in range(len(n))]
    P = T.ts_plan_create(n, L, f, mask, order=k)
    Po0 = sem.plan(n, L, [np.zeros(m) for m in n], k)
    PoV = sem.plan(n, L, f, k)
    return P, Po0, PoV, sem.potential_sum(PoV).reshape(-1)


@pytest.mark.parametrize("n,k,L", [((29, 19, 39), 10, (5.0, 4.0, 6.0)), ((24, 17, 9), 1, (4.0, 3.0, 2.5))])
def test_h1_flow_steps_vs_oracle(T, n, k, L):
    P, Po0, PoV, V = _case(T, n, k, L)
    beta, steps = 30.0, 25
    u0 = np.cos(0.3 * np.arange(Po0.N)) + 1.5
    uo = gpe.normalize(Po0, u0)
    for _ in range(steps):
        uo = gpe.h1_flow_step(Po0, V, beta, 20.0, 0.1, uo)
    u = dev(u0)
    E, lam, it, solves, _ = T.ts_gpe_ground_state(P, None, beta, T.TS_GPE_H1, u, 20.0, 0.1, 0.0, 0.0, steps,
                                                  allow_not_converged=True)
    assert it == steps and solves == 2 * steps
    assert rel(host(u), uo) < 1e-10
    assert abs(E - gpe.energy(Po0, V, beta, uo)) < 1e-12 * abs(E)
    assert abs(lam - gpe.eigenvalue(Po0, V, beta, uo)) < 1e-12 * abs(lam)


def test_au_flow_steps_vs_oracle(T):
    n, k, L = (29, 19, 39), 10, (5.0, 4.0, 6.0)
    P, Po0, PoV, V = _case(T, n, k, L)
    beta, steps = 30.0, 6
    u0 = np.cos(0.3 * np.arange(PoV.N)) + 1.5
    uo = gpe.normalize(PoV, u0)
    for _ in range(steps):
        uo = gpe.au_flow_step(PoV, V, beta, 1.0, uo, pcg_tol=1e-13)
    u = dev(u0)
    E, lam, it, solves, _ = T.ts_gpe_ground_state(P, None, beta, T.TS_GPE_AU, u, 0.0, 1.0, 0.0, 0.0, steps,
                                                  pcg_tol=1e-13, allow_not_converged=True)
    assert it == steps and solves > steps
    assert rel(host(u), uo) < 1e-9
    assert abs(E - gpe.energy(PoV, V, beta, uo)) < 1e-12 * abs(E)


def test_split_precision_g_reaches_the_fp64_minimiser(T):
    """G applied by the BF16X3 tensor-core inverse with two FP64-residual refinements: the
    flow converges to the same minimiser as with the FP64 inverse (the fixed point does not
    depend on G); converged on the Euler-Lagrange residual."""
    n, k, L = (29, 19, 39), 10, (5.0, 4.0, 6.0)
    P, _, _, _ = _case(T, n, k, L, mask=1 << T.TS_BF16X3)
    N = int(np.prod(n))
    out = []
    for prec in (T.TS_FP64, T.TS_BF16X3):
        u = dev(np.ones(N))
        out.append(T.ts_gpe_ground_state(P, None, 30.0, T.TS_GPE_H1, u, 20.0, 0.1, 0.0, 1e-11, 5000, prec) + (u,))
    assert abs(out[0][0] - out[1][0]) < 1e-13 * out[0][0]
    assert abs(out[0][1] - out[1][1]) < 1e-10 * out[0][1]
    assert rel(host(out[1][5]), host(out[0][5])) < 1e-9


def _paper_grid(T, n, mask=0):
    import torch
    k, L = 20, 8.0
    x, _ = T.ts_grid_nodes(n, L, k)
    f1 = x ** 2 + 100 * np.sin(np.pi * x / 4) ** 2
    P = T.ts_plan_create((n,) * 3, (L,) * 3, [f1] * 3, mask, order=k)
    g = torch.from_numpy(T.ts_plan_eigvecs(P, 0)[:, 0].copy()).cuda()  # the 1D linear ground state
    u0 = (g[:, None, None] * g[None, :, None] * g[None, None, :]).reshape(-1).contiguous()
    return P, u0


@pytest.mark.parametrize("beta,E_printed,lam_printed,prec", [(10.0, 14.1965761916, 32.4916917439, "fp64"),
                                                             (100.0, 20.6824463703, 47.7831207152, "bf16x3")])
def test_paper_table_h1_flow(T, beta, E_printed, lam_printed, prec):
    """Table h1_flow: modified H^1 flow, alpha = 20, tau = 0.1, from the linear ground state
    of -Delta + V1 (V1 = sum (x_k^2 + 100 sin^2(pi x_k / 4))), Q^20 on [-8, 8]^3: energy and
    eigenvalue to the printed digits.  n = 199 per axis: the linear ground state is then
    converged to 4e-11 (the 1D oracle), the table used 599."""
    p = T.TS_FP64 if prec == "fp64" else T.TS_BF16X3
    P, u0 = _paper_grid(T, 199, 0 if prec == "fp64" else 1 << T.TS_BF16X3)
    u = u0.clone()
    # the table's stopping rule (energy change below 1e-14): the energy, and the step count
    E, lam, it, _, res = T.ts_gpe_ground_state(P, None, beta, T.TS_GPE_H1, u, 20.0, 0.1, 1e-14, 0.0, 2000, p)
    assert abs(E - E_printed) < 1e-9
    print(f"beta {beta}: {it} steps to |dE|/E < 1e-14 (table at 599^3: 175 / 405), residual {res:.2e}")
    # continued until the Euler-Lagrange residual bounds the error of lambda
    E, lam, it2, _, res = T.ts_gpe_ground_state(P, None, beta, T.TS_GPE_H1, u, 20.0, 0.1, 0.0, 1e-11, 20000, p)
    print(f"beta {beta}: lambda {lam!r} after {it2} more steps, residual {res:.2e}")
    assert abs(E - E_printed) < 1e-9 and abs(lam - lam_printed) < 1e-8


@pytest.mark.parametrize("flow,tau,steps_printed,solves_printed", [("au", 1.0, 66, 790), ("h1", 0.1, 272, 544)])
def test_paper_table_au_vs_h1_beta1600(T, flow, tau, steps_printed, solves_printed):
    """Table au_vs_h1: beta = 1600, constant initial guess, Q^20 on [-8, 8]^3, V1 of eq.
    separable_V1, alpha = 20; a_u with tau = 1 and PCG (preconditioner (-Delta + V1)^{-1},
    tolerance 1e-12), modified H^1 with tau = 0.1, both until |E_k - E*| / E* < 1e-12 with
    E* = 33.80227900547423 (the table's criterion).  n = 199 (the table: 599) already reaches
    E* to that tolerance; the step and linear-solve counts agree with the table's within
    15% (a_u: 66 steps, 790 PCG iterations; H^1: 272 steps, 544 direct solves)."""
    import torch
    Estar = 33.80227900547423
    P, _ = _paper_grid(T, 199, 1 << T.TS_BF16X3)
    u = torch.ones(P.N, dtype=torch.float64, device="cuda")
    f = T.TS_GPE_AU if flow == "au" else T.TS_GPE_H1
    steps = solves = 0
    while True:  # in chunks of 5 steps, to apply the table's criterion with E* known
        E, lam, it, so, _ = T.ts_gpe_ground_state(P, None, 1600.0, f, u, 20.0, tau, 0.0, 0.0, 5, T.TS_BF16X3,
                                                  pcg_tol=1e-12, allow_not_converged=True)
        steps, solves = steps + it, solves + so
        if abs(E - Estar) < 1e-12 * Estar or steps > 2000:
            break
    print(f"{flow}: {steps} steps, {solves} solves, E = {E!r}")
    assert abs(E - Estar) < 1e-12 * Estar
    assert abs(steps - steps_printed) <= 0.15 * steps_printed
    assert abs(solves - solves_printed) <= 0.15 * solves_printed
