"""Parity of the FP64 CUDA path with the CPU oracle, element by element, through the C ABI.

Sizes span several CUDA tiles and leave ragged tails (n not a multiple of the tile);
tolerance 1e-12 relative l2 for every FP64 path."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import dev, harmonic_case, host, plans, rel

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


@pytest.mark.parametrize("n", [(32, 32, 32), (70, 33, 9), (5,), (17, 130), (8, 7, 6, 5)])
def test_plan_eigenvalues_match_oracle(T, n):
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    for k in range(len(n)):
        lam = T.ts_plan_eigs(P, k)
        assert np.max(np.abs(lam - Po.lam[k])) < 1e-13 * np.abs(Po.lam[k]).max()
        S_ = T.ts_plan_eigvecs(P, k)
        assert np.max(np.abs(S_.T @ S_ - np.eye(n[k]))) < 1e-13


def test_config1_inverse_vs_oracle_and_dense_lu(T):
    """3D n = 32 on [-8,8]^3, V1 = sum x^2, sigma = 1, b ~ U[-1,1) seed 0; dense LU at n = 8."""
    w = S.WORKLOADS["3d_n32_fp64"]
    for n in (w["n"], (w["lu_n"],) * 3):
        L, f = w["L"], S.harmonic(n, w["L"], w["omega"])
        P, Po = plans(n, L, f)
        b = S.uniform(w["seed"], Po.N)
        u = dev(np.zeros(Po.N))
        T.ts_apply_inverse(P, w["sigma"], dev(b), u)
        got = host(u)
        assert rel(got, O.apply_inverse(Po, w["sigma"], b)) < TOL
        if n[0] == w["lu_n"]:
            assert rel(got, O.lu_solve(O.dense_operator(Po, w["sigma"]), b)) < TOL


@pytest.mark.parametrize("n", [(70, 33, 9), (100, 65), (3, 4, 5, 6, 2), (129,), (24, 24, 24, 8)])
def test_inverse_ragged_shapes(T, n):
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    b = S.normal(5, Po.N)
    bt = dev(b)
    T.ts_apply_inverse(P, 0.7, bt, bt)  # in place (b and u alias)
    assert rel(host(bt), O.apply_inverse(Po, 0.7, b)) < TOL


@pytest.mark.parametrize("n", [(20, 18, 16), (6, 6, 6, 6, 6, 6), (3,) * 9, (65, 40)])
def test_exp_c128_vs_oracle(T, n):
    L, f = harmonic_case(n, L=4.0)
    P, Po = plans(n, L, f)
    psi = S.complex_normal(3, Po.N)
    out = dev(np.zeros(2 * Po.N))
    T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C128)
    want = O.apply_exp(Po, 0.01, psi)
    assert rel(host(out), want) < TOL


def test_exp_c64_data_fp64_arithmetic(T):
    n = (12, 10, 14)
    L, f = harmonic_case(n, L=4.0)
    P, Po = plans(n, L, f)
    psi = S.complex_normal(3, Po.N).astype(np.float32)
    out = dev(np.zeros(2 * Po.N, dtype=np.float32))
    T.ts_apply_exp(P, 0.05, dev(psi), out, T.TS_C64)
    want = O.apply_exp(Po, 0.05, psi.astype(np.float64))
    assert rel(host(out), want) < 1e-6  # input/output rounding to complex64


def test_operator_stencil_vs_oracle(T):
    n = (30, 17, 9)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    x = S.normal(1, Po.N)
    V2 = S.uniform(2, Po.N, 0, 3)
    y = dev(np.zeros(Po.N))
    T.ts_apply_operator(P, 0.3, dev(V2), dev(x), y)
    assert rel(host(y), O.stencil(Po, x, 0.3, V2)) < 1e-14


def test_pcg_fp64_vs_oracle(T):
    n = (40, 36, 33)
    L, f = harmonic_case(n, omega=(1, 1, 1))
    P, Po = plans(n, L, f)
    V2 = S.v2_cos_bumps(n, L, seed=1) + 5.0
    b = S.uniform(0, Po.N)
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 0.0, 0.0, dev(V2), dev(b), x, 1e-12, 200)
    xo, ito, _ = O.pcg(Po, b, sigma=0.0, V2=V2, tol=1e-12)
    assert relres < 1e-11
    assert abs(it - ito) <= 1
    assert rel(host(x), xo) < 1e-11


def test_pcg_trivial_cases(T):
    n = (16, 16, 16)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    b = S.uniform(0, Po.N)
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 1.0, 1.0, None, dev(b), x, 1e-12, 10)
    assert it == 1 and relres < 1e-13
    V2 = np.full(Po.N, 2.5)
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 1.0, 3.5, dev(V2), dev(b), x, 1e-12, 10)
    assert it == 1 and relres < 1e-13
    # zero right-hand side: nothing to do
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 1.0, 1.0, None, dev(np.zeros(Po.N)), x, 1e-12, 10)
    assert it == 0


def test_inverse_iteration_vs_oracle(T):
    n = (24, 24, 24)
    L, f = harmonic_case(n, omega=(1, 1, 1))
    P, Po = plans(n, L, f)
    V2 = S.v2_cos_bumps(n, L, seed=1)
    s = sum(l[0] for l in Po.lam) + V2.min() - 1.0
    u = dev(np.zeros(Po.N))
    lam, outer, tot = T.ts_inverse_iteration(P, s, dev(V2), u, True, 1e-12, 300, 1e-10, 500)
    uo, lamo, ito, toto = O.inverse_iteration(Po, s, V2, tol_lambda=1e-12, maxit=300, pcg_tol=1e-10)
    assert abs(lam - lamo) / abs(lamo) < 1e-11
    assert abs(outer - ito) <= 1
    assert np.linalg.norm(host(u) - uo) < 1e-5


def test_inverse_iteration_on_poisoned_scratch(T):
    """Scratch buffers come back from the pool with whatever the last user left in them:
    here the pool is filled with NaNs by an FP64 apply of a NaN right-hand side first.  The
    warm start w_0 = u / (lambda - s) must not read the old contents of w (0 * NaN = NaN)."""
    n = (24, 24, 24)
    L, f = harmonic_case(n, omega=(1, 1, 1))
    P, Po = plans(n, L, f)
    junk = dev(np.full(Po.N, np.nan))
    out = dev(np.zeros(Po.N))
    for _ in range(3):
        T.ts_apply_inverse(P, 0.5, junk, out)  # leaves NaN in the pool's buffers
    V2 = S.v2_cos_bumps(n, L, seed=1)
    s = sum(l[0] for l in Po.lam) + V2.min() - 1.0
    u = dev(np.zeros(Po.N))
    lam, outer, tot = T.ts_inverse_iteration(P, s, dev(V2), u, True, 1e-12, 300, 1e-10, 500)
    uo, lamo, ito, toto = O.inverse_iteration(Po, s, V2, tol_lambda=1e-12, maxit=300, pcg_tol=1e-10)
    assert np.isfinite(lam) and abs(lam - lamo) / abs(lamo) < 1e-11


@pytest.mark.parametrize("n,dtype", [((6,) * 6, "c128"), ((3,) * 9, "c128"), ((6,) * 6, "c64")])
def test_strang_vs_oracle(T, n, dtype):
    d = len(n)
    Lv = 5.0 if d == 6 else 3.0
    L = (Lv,) * d
    f = S.harmonic(n, L, (1.0,) * d)
    P, Po = plans(n, L, f)
    V2 = S.v2_soft_coulomb(n, L)
    psi = S.sine_state(n, L)
    want = O.strang(Po, V2, 0.01, 10, psi)
    if dtype == "c128":
        t = dev(psi)
        T.ts_split_step(P, 0.01, 10, dev(V2), t, T.TS_C128)
        assert rel(host(t), want) < TOL
    else:
        t = dev(psi.astype(np.float32))
        T.ts_split_step(P, 0.01, 10, dev(V2), t, T.TS_C64)
        assert rel(host(t), want) < 1e-6


@pytest.mark.parametrize("n", [(40, 24, 56), (33, 33, 33), (64, 16, 40)])
def test_pcg_fixed_point_operator_vs_oracle(T, n):
    """On grids with one spacing h (d = 3) PCG applies A in exact fixed point (Laplacian and
    sigma + V1 as one integer sum, V2 x in FP64): same iterate as the oracle's textbook PCG,
    on ragged tiles, with a mixed (BF16X3) preconditioner too."""
    L = tuple((k + 1) / 4.0 for k in n)
    f = S.harmonic(n, L, (1.0, 1.2, 0.8))
    P = T.ts_plan_create(n, L, f, 1 << T.TS_BF16X3)
    Po = O.plan(n, L, f)
    V2 = S.v2_cos_bumps(n, L, seed=1) + 5.0
    b = S.uniform(0, Po.N)
    xo, ito, _ = O.pcg(Po, b, sigma=0.3, V2=V2, tol=1e-12)
    for prec in (T.TS_FP64, T.TS_BF16X3):
        x = dev(np.zeros(Po.N))
        st, it, relres = T.ts_pcg(P, 0.3, 0.3, dev(V2), dev(b), x, 1e-12, 200, prec)
        assert relres < 1e-11
        assert rel(host(x), xo) < 1e-10
        if prec == T.TS_FP64:
            assert abs(it - ito) <= 1


@pytest.mark.parametrize("n", [(40, 24, 56), (33, 33, 33)])
def test_operator_fixed_point_vs_oracle(T, n):
    """ts_apply_operator on grids with one spacing (d = 3): the exact fixed-point form agrees
    with the oracle's FP64 stencil to rounding, also for x spanning eleven decades."""
    L = tuple((k + 1) / 4.0 for k in n)
    f = S.harmonic(n, L, (1.0, 1.2, 0.8))
    P = T.ts_plan_create(n, L, f, 0)
    Po = O.plan(n, L, f)
    V2 = S.uniform(2, Po.N, 0, 3)
    for x in (S.normal(1, Po.N), S.normal(1, Po.N) * np.exp(S.uniform(3, Po.N, -12.0, 13.0))):
        y = dev(np.zeros(Po.N))
        T.ts_apply_operator(P, 0.3, dev(V2), dev(x), y)
        assert rel(host(y), O.stencil(Po, x, 0.3, V2)) < 1e-14


def test_axis_tables_evicted_and_reused(T):
    """More distinct axes than the process-wide axis cache keeps (128): 60 plans of three
    fresh axes each (Q^1, host tridiagonal QR), each destroyed after use, so evicted tables
    go back to the table pool and later plans reuse their memory.  Every plan's FP64 and
    BF16X3 inverse still matches the oracle, and two plans built on identical axes (one
    before and one after the evictions) give identical results."""
    n, L = (12, 9, 7), (8.0, 8.0, 8.0)
    rng = np.random.default_rng(11)
    b = S.normal(3, int(np.prod(n)))
    f_first = None
    u_first = None
    for i in range(60):
        om = tuple(rng.uniform(0.5, 2.0, 3))
        f = S.harmonic(n, L, om)
        if i == 0:
            f_first = f
        P, Po = plans(n, L, f, 1 << T.TS_BF16X3)
        u = dev(np.zeros(Po.N))
        T.ts_apply_inverse(P, 0.7, dev(b), u)
        if i == 0:
            u_first = host(u)
        if i % 6 == 0:
            ref = O.apply_inverse(Po, 0.7, b)
            assert rel(host(u), ref) < TOL
            T.ts_apply_inverse(P, 0.7, dev(b), u, T.TS_BF16X3)
            assert rel(host(u), ref) < 1e-4
        T.ts_plan_destroy(P)
    P = T.ts_plan_create(n, L, f_first, 0)
    u = dev(np.zeros(int(np.prod(n))))
    T.ts_apply_inverse(P, 0.7, dev(b), u)
    assert np.array_equal(host(u), u_first)
