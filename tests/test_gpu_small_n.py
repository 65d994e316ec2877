"""The FP32 fused small-n path (complex64, n_k in {8, 16, 24, 32}) against the oracle, and
the full-size 6D / 9D Strang workloads against the FP64 GPU path and the unitarity of the
propagator.  FP32 tolerance: each mode contraction rounds O(sqrt(n) 2^-24); 2d modes per
apply stay below 2e-6 and 10 Strang steps below 1e-5."""
import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import MAXNORM_FACTOR, dev, host, maxrel, plans, rel

pytestmark = pytest.mark.gpu
FP32_MASK = 1 << 5


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


@pytest.mark.parametrize("n", [(24, 24, 24), (8,) * 5, (16,) * 4, (32, 8, 24), (8,) * 7])
def test_fp32_exp_vs_oracle(T, n):
    d = len(n)
    L = (4.0,) * d
    f = S.harmonic(n, L, tuple(1.0 + 0.1 * k for k in range(d)))
    P, Po = plans(n, L, f, FP32_MASK)
    psi = S.complex_normal(3, Po.N).astype(np.float32)
    out = dev(np.zeros(2 * Po.N, dtype=np.float32))
    T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C64, T.TS_FP32)
    got = host(out).astype(np.float64)
    want = O.apply_exp(Po, 0.01, psi.astype(np.float64))
    err = rel(got, want)
    assert err < 2e-6, err
    assert maxrel(got, want) < MAXNORM_FACTOR * 2e-6
    # in place
    x = dev(psi)
    T.ts_apply_exp(P, 0.01, x, x, T.TS_C64, T.TS_FP32)
    assert np.array_equal(host(x), host(out))


@pytest.mark.parametrize("n,Lv", [((8,) * 6, 5.0), ((16, 16, 16), 3.0), ((8,) * 9, 3.0)])
def test_fp32_strang_vs_oracle(T, n, Lv):
    d = len(n)
    L = (Lv,) * d
    f = S.harmonic(n, L, (1.0,) * d)
    P, Po = plans(n, L, f, FP32_MASK)
    V2 = S.v2_soft_coulomb(n, L)
    psi = S.sine_state(n, L)
    steps = 10 if Po.N <= 300000 else 2
    want = O.strang(Po, V2, 0.01, steps, psi)
    t = dev(psi.astype(np.float32))
    T.ts_split_step(P, 0.01, steps, dev(V2), t, T.TS_C64, T.TS_FP32)
    got = host(t).astype(np.float64)
    assert rel(got, want) < 1e-5
    assert maxrel(got, want) < MAXNORM_FACTOR * 1e-5


@pytest.mark.parametrize("name", ["6d_n24_strang", "9d_n8_strang"])
def test_full_size_strang_fp32_vs_fp64_path(T, name):
    """The high-d workloads at full size (1.9e8 / 1.3e8 DoF), 100 steps: complex64 FP32 fused
    path against the complex128 FP64 path on the GPU (itself oracle-checked at small
    sizes), and norm preservation of both."""
    import torch
    w = S.WORKLOADS[name]
    n, L = w["n"], w["L"]
    f = S.harmonic(n, L, w["omega"])
    P = T.ts_plan_create(n, L, f, FP32_MASK)
    V2 = dev(S.v2_soft_coulomb(n, L))
    psi0 = S.sine_state(n, L)
    a = dev(psi0.astype(np.float32))
    T.ts_split_step(P, w["dt"], w["steps"], V2, a, T.TS_C64, T.TS_FP32)
    b = dev(psi0)
    T.ts_split_step(P, w["dt"], w["steps"], V2, b, T.TS_C128, T.TS_FP64)
    a64 = a.double()
    d = ((a64 - b).norm() / b.norm()).item()
    assert d < 1e-4, d
    assert abs(a64.norm().item() - 1.0) < 1e-4
    assert abs(b.norm().item() - 1.0) < 1e-12
    del a, b, a64
    torch.cuda.empty_cache()


def test_full_size_6d_strang_two_steps_vs_oracle(T):
    """The 6D workload at its full size (24^6 = 1.9e8 DoF): two complex64 Strang steps of
    the FP32 path against the oracle's unmerged FP64 Strang steps (forward transforms,
    phase, backward transforms and half-step potential phases, plain loops)."""
    w = S.WORKLOADS["6d_n24_strang"]
    n, L = w["n"], w["L"]
    f = S.harmonic(n, L, w["omega"])
    P, Po = plans(n, L, f, FP32_MASK)
    V2 = S.v2_soft_coulomb(n, L)
    psi = S.sine_state(n, L)
    t = dev(psi.astype(np.float32))
    T.ts_split_step(P, w["dt"], 2, dev(V2), t, T.TS_C64, T.TS_FP32)
    got = host(t).astype(np.float64)
    del t
    want = O.strang(Po, V2, w["dt"], 2, psi)
    assert rel(got, want) < 1e-5
    assert maxrel(got, want) < MAXNORM_FACTOR * 1e-5
