"""ts_propagate (Sec. 5.1 splittings) on the GPU, through the C ABI.

The library merges adjacent propagations (Remark cost_naive_merged); the oracle applies the
product formula factor by factor (oracle/splitting.py), so agreement to rounding checks the
merge.  Then Table splitting's Delta t = 0.1 row at the table's full 499^3 Q^10 grid."""
import numpy as np
import pytest

import oracle as O
from oracle import sem
from oracle import splitting as SP
from paper_2605_20491_b300 import synth as S
from gpu_util import dev, harmonic_case, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def _q1_case(T, n, mask=0):
    L, f = harmonic_case(n, L=4.0)
    P = T.ts_plan_create(n, L, f, mask)
    Po = O.plan(n, L, f)
    expA = lambda t, p: O.apply_exp(Po, t, np.ascontiguousarray(p).view(np.float64)).view(np.complex128)  # noqa: E731
    return P, Po.N, expA


def _qk_case(T, n, k, mask=0):
    L = tuple(2.0 + 0.5 * a for a in range(len(n)))
    f = [0.5 * sem.axis_1d(n[a], L[a], k).x ** 2 for a in range(len(n))]
    P = T.ts_plan_create(n, L, f, mask, order=k)
    Po = sem.plan(n, L, f, k)
    return P, Po.N, lambda t, p: sem.apply_exp(Po, t, p)


SCHEMES = [("strang", 1), ("qhop", 1), ("qhop", 3), ("qhop", 5), ("magnus2", 1), ("magnus2", 3)]


def _scheme(T, name):
    return {"strang": T.TS_STRANG, "qhop": T.TS_QHOP, "magnus2": T.TS_MAGNUS2}[name]


def _expected_props(name, M, nsteps):
    if name == "strang" or (name == "qhop" and M == 1):
        return nsteps
    if name == "qhop":
        return nsteps * M + 1
    return 3 * nsteps if M == 1 else 3 * nsteps * M + 1


@pytest.mark.parametrize("name,M", SCHEMES)
@pytest.mark.parametrize("grid", ["q1", "q3"])
def test_schemes_fp64_vs_unmerged_oracle(T, name, M, grid):
    P, N, expA = _q1_case(T, (24, 17, 9)) if grid == "q1" else _qk_case(T, (11, 14, 8), 3)
    rng = np.random.default_rng(3)
    VB = rng.uniform(0, 4, N)
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi /= np.linalg.norm(psi)
    expB = lambda t, p: np.exp(-1j * t * VB) * p  # noqa: E731
    dt, nsteps = 0.02, 3
    want = SP.propagate("magnus2" if name == "magnus2" else "qhop", M, dt, nsteps, psi, expA, expB)
    x = dev(psi.view(np.float64))
    na = T.ts_propagate(P, _scheme(T, name), M, dt, nsteps, dev(VB), x, T.TS_C128)
    assert na == _expected_props(name, M, nsteps)
    assert rel(host(x).view(np.complex128), want) < 1e-11


def test_schemes_split_precision_and_fp32(T):
    """The same schemes on the BF16X3 tensor-core propagator (complex128 data) and on the
    FP32 fused small-n propagator (complex64), against the FP64 oracle: each
    A-propagation adds its precision's error (BF16X3 ~1e-5, FP32 ~1e-6)."""
    n = (16, 8, 24)
    P, N, expA = _q1_case(T, n, (1 << T.TS_BF16X3) | (1 << T.TS_FP32))
    rng = np.random.default_rng(4)
    VB = rng.uniform(0, 4, N)
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi /= np.linalg.norm(psi)
    expB = lambda t, p: np.exp(-1j * t * VB) * p  # noqa: E731
    for name, M in (("qhop", 3), ("magnus2", 1)):
        want = SP.propagate(name, M, 0.02, 2, psi, expA, expB)
        x = dev(psi.view(np.float64))
        na = T.ts_propagate(P, _scheme(T, name), M, 0.02, 2, dev(VB), x, T.TS_C128, T.TS_BF16X3)
        assert rel(host(x).view(np.complex128), want) < 5e-5 * na
        x = dev(psi.astype(np.complex64).view(np.float32))
        na = T.ts_propagate(P, _scheme(T, name), M, 0.02, 2, dev(VB), x, T.TS_C64, T.TS_FP32)
        assert rel(host(x).view(np.complex64), want) < 2e-6 * na


def test_strang_equals_split_step(T):
    """TS_STRANG is the merged B-A-B Strang of ts_split_step."""
    import torch
    n = (24, 17, 9)
    P, N, _ = _q1_case(T, n)
    VB = dev(S.uniform(5, N, 0.0, 3.0))
    psi = dev(S.complex_normal(6, N))
    a, b = psi.clone(), psi.clone()
    T.ts_propagate(P, T.TS_STRANG, 1, 0.03, 4, VB, a, T.TS_C128)
    T.ts_split_step(P, 0.03, 4, VB, b, T.TS_C128)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_propagate_rejects_bad_arguments(T):
    P, N, _ = _q1_case(T, (8, 8))
    x = dev(np.zeros(2 * N))
    VB = dev(np.zeros(N))
    for scheme, M in ((7, 1), (T.TS_QHOP, 0), (T.TS_QHOP, 65)):
        with pytest.raises(T.TsError):
            T.ts_propagate(P, scheme, M, 0.01, 1, VB, x, T.TS_C128)
    assert T.ts_propagate(P, T.TS_QHOP, 3, 0.01, 0, VB, x, T.TS_C128) == 0


def test_paper_table_splitting_dt01_full_size(T):
    """Table splitting, Delta t = 0.1 row (one step to T = 0.1), at the table's grid: Q^10,
    499^3 DoFs on [-8, 8]^3, complex128 in FP64, A = -Delta (plan with f = 0),
    B = V1 = sum_k (x_k^2 + 100 sin^2(pi x_k / 4)), psi_0 = prod sin(pi (x_k + L) / 2L)
    normalised, reference = the exact propagator of the plan with V1.  Printed errors:
    5.85e-1 (M = 1, Strang), 1.07e-1 (3), 4.25e-2 (5), 2.28e-2 (7)."""
    import torch
    n, k, L = 499, 10, 8.0
    x, _ = T.ts_grid_nodes(n, L, k)
    v1 = x ** 2 + 100 * np.sin(np.pi * x / 4) ** 2
    PA = T.ts_plan_create((n,) * 3, (L,) * 3, [np.zeros(n)] * 3, 0, order=k)
    PH = T.ts_plan_create((n,) * 3, (L,) * 3, [v1] * 3, 0, order=k)
    xs = torch.from_numpy(x).cuda()
    s1 = torch.sin(np.pi * (xs + L) / (2 * L))
    psi0 = (s1[:, None, None] * s1[None, :, None] * s1[None, None, :]).reshape(-1)
    psi0 = (psi0 / torch.linalg.vector_norm(psi0)).to(torch.complex128)
    v = torch.from_numpy(v1).cuda()
    VB = (v[:, None, None] + v[None, :, None] + v[None, None, :]).reshape(-1).contiguous()
    ref = torch.empty_like(psi0)
    T.ts_apply_exp(PH, 0.1, torch.view_as_real(psi0), torch.view_as_real(ref), T.TS_C128)
    for M, printed in ((1, 5.85e-1), (3, 1.07e-1), (5, 4.25e-2), (7, 2.28e-2)):
        psi = psi0.clone()
        T.ts_propagate(PA, T.TS_QHOP, M, 0.1, 1, VB, torch.view_as_real(psi), T.TS_C128)
        err = torch.linalg.vector_norm(psi - ref).item()
        assert abs(err - printed) <= 0.0051 * printed, (M, err)
