"""The small-n route of TS_BF16X6 on complex64 against the oracle: axes of 16 or 24 points
two per pass on the tensor cores, 8-point axes on the FP32 kernels.  On the tensor cores
each axis is a real 2n x 2n product split into three bf16 planes (six products: every
term above 2^-24 relative kept); the leading product accumulates alone in FP32, so the
error of one axis is the FP32 accumulation of 2n terms plus the FP32 rounding of the
result and its re-split, O(2n 2^-24) relative at worst.  With d <= 9 axes per apply this
stays below 5e-6; 10 Strang steps below 3e-5.  The cases cover tiles along the lower axes
(lo > 1), along the upper ones (lo = 1), groups that go to the FFMA kernels (a single
axis, 8-point axes, or a tile dimension 16 does not divide) and mixed lengths."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import MAXNORM_FACTOR, dev, host, maxrel, plans, rel

pytestmark = pytest.mark.gpu
X6_MASK = 1 << 2
EXP_TOL = 5e-6
STRANG_TOL = 3e-5


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


@pytest.mark.parametrize("n", [(24,) * 4, (16,) * 4, (16, 24, 24, 16), (24,) * 5, (16,) * 3, (24, 24), (16,) * 6,
                               (8,) * 6, (8,) * 5, (8,) * 7, (8,) * 3, (8, 8, 8, 16, 16)])
def test_bf16x6_exp_vs_oracle(T, n):
    d = len(n)
    L = (4.0,) * d
    f = S.harmonic(n, L, tuple(1.0 + 0.1 * k for k in range(d)))
    P, Po = plans(n, L, f, X6_MASK)
    psi = S.complex_normal(7, Po.N).astype(np.float32)
    out = dev(np.zeros(2 * Po.N, dtype=np.float32))
    T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C64, T.TS_BF16X6)
    T.ts_device_status()  # raises if a bounded wait gave up
    got = host(out).astype(np.float64)
    want = O.apply_exp(Po, 0.01, psi.astype(np.float64))
    err = rel(got, want)
    assert err < EXP_TOL, err
    assert maxrel(got, want) < MAXNORM_FACTOR * EXP_TOL
    # in place gives the same bits (tiles are disjoint, each read before it is written)
    x = dev(psi)
    T.ts_apply_exp(P, 0.01, x, x, T.TS_C64, T.TS_BF16X6)
    assert np.array_equal(host(x), host(out))


def test_bf16x6_exp_large_tau_is_unitary(T):
    """tau = 1 (phases of many turns): the propagator is unitary to the working accuracy and
    matches the oracle."""
    n = (24,) * 4
    L = (4.0,) * 4
    f = S.harmonic(n, L, (1.0,) * 4)
    P, Po = plans(n, L, f, X6_MASK)
    psi = S.complex_normal(11, Po.N).astype(np.float32)
    out = dev(np.zeros(2 * Po.N, dtype=np.float32))
    T.ts_apply_exp(P, 1.0, dev(psi), out, T.TS_C64, T.TS_BF16X6)
    got = host(out).astype(np.float64)
    want = O.apply_exp(Po, 1.0, psi.astype(np.float64))
    assert rel(got, want) < EXP_TOL
    assert abs(np.linalg.norm(got) / np.linalg.norm(psi.astype(np.float64)) - 1.0) < EXP_TOL


@pytest.mark.parametrize("n,Lv,steps,dim", [((16,) * 4, 3.0, 10, 2), ((24,) * 4, 5.0, 4, 2), ((16, 16, 16), 3.0, 10, 3),
                                            ((8,) * 6, 5.0, 10, 3)])
def test_bf16x6_strang_vs_oracle(T, n, Lv, steps, dim):
    """Two particles in 2D (d = 4) or one in 3D, soft-Coulomb V2: the phases folded into the
    first and last pass of each step, across tiles along the lower and upper axes."""
    d = len(n)
    L = (Lv,) * d
    f = S.harmonic(n, L, (1.0,) * d)
    P, Po = plans(n, L, f, X6_MASK)
    V2 = S.v2_soft_coulomb(n, L, dim=dim)
    psi = S.sine_state(n, L)
    want = O.strang(Po, V2, 0.01, steps, psi)
    t = dev(psi.astype(np.float32))
    T.ts_split_step(P, 0.01, steps, dev(V2), t, T.TS_C64, T.TS_BF16X6)
    got = host(t).astype(np.float64)
    assert rel(got, want) < STRANG_TOL
    assert maxrel(got, want) < MAXNORM_FACTOR * STRANG_TOL


@functools.lru_cache(maxsize=1)
def _oracle_6d_two_steps():
    w = S.WORKLOADS["6d_n24_strang"]
    n, L = w["n"], w["L"]
    Po = O.plan(n, L, S.harmonic(n, L, w["omega"]))
    return O.strang(Po, S.v2_soft_coulomb(n, L), w["dt"], 2, S.sine_state(n, L))


def test_full_size_6d_bf16x6_two_steps_vs_oracle(T):
    """The 6D workload at full size (24^6 = 1.9e8 DoF): two Strang steps of the tensor-core
    pass against the oracle's unmerged FP64 Strang steps."""
    import torch
    w = S.WORKLOADS["6d_n24_strang"]
    n, L = w["n"], w["L"]
    P = T.ts_plan_create(n, L, S.harmonic(n, L, w["omega"]), X6_MASK)
    t = dev(S.sine_state(n, L).astype(np.float32))
    T.ts_split_step(P, w["dt"], 2, dev(S.v2_soft_coulomb(n, L)), t, T.TS_C64, T.TS_BF16X6)
    T.ts_device_status()  # raises if a bounded wait gave up
    got = host(t).astype(np.float64)
    del t
    torch.cuda.empty_cache()
    want = _oracle_6d_two_steps()
    assert rel(got, want) < STRANG_TOL
    assert maxrel(got, want) < MAXNORM_FACTOR * STRANG_TOL


def test_full_size_6d_bf16x6_100_steps_vs_fp64_path(T):
    """100 steps of the full-size workload: the tensor-core pass against the complex128 FP64
    path on the GPU, and norm preservation."""
    import torch
    w = S.WORKLOADS["6d_n24_strang"]
    n, L = w["n"], w["L"]
    f = S.harmonic(n, L, w["omega"])
    P = T.ts_plan_create(n, L, f, X6_MASK | 1)
    V2 = dev(S.v2_soft_coulomb(n, L))
    psi0 = S.sine_state(n, L)
    a = dev(psi0.astype(np.float32))
    T.ts_split_step(P, w["dt"], w["steps"], V2, a, T.TS_C64, T.TS_BF16X6)
    b = dev(psi0)
    T.ts_split_step(P, w["dt"], w["steps"], V2, b, T.TS_C128, T.TS_FP64)
    a64 = a.double()
    dlt = ((a64 - b).norm() / b.norm()).item()
    assert dlt < 1e-4, dlt
    assert abs(a64.norm().item() - 1.0) < 1e-4
    del a, b, a64
    torch.cuda.empty_cache()


def test_full_size_9d_bf16x6_two_steps_vs_oracle(T):
    """The 9D workload at full size (8^9 = 1.3e8 DoF) requested in TS_BF16X6: two Strang
    steps (the FP32 three-axis kernels serve 8-point axes) against the oracle's unmerged
    FP64 Strang steps."""
    import torch
    w = S.WORKLOADS["9d_n8_strang"]
    n, L = w["n"], w["L"]
    P, Po = plans(n, L, S.harmonic(n, L, w["omega"]), X6_MASK)
    V2 = S.v2_soft_coulomb(n, L)
    psi = S.sine_state(n, L)
    t = dev(psi.astype(np.float32))
    T.ts_split_step(P, w["dt"], 2, dev(V2), t, T.TS_C64, T.TS_BF16X6)
    T.ts_device_status()  # raises if a bounded wait gave up
    got = host(t).astype(np.float64)
    del t
    torch.cuda.empty_cache()
    want = O.strang(Po, V2, w["dt"], 2, psi)
    assert rel(got, want) < STRANG_TOL
    assert maxrel(got, want) < MAXNORM_FACTOR * STRANG_TOL
