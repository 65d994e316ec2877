"""Failure detection without a GPU fault: bounded device waits that run out and report,
iteration caps, non-finite input, invalid handles and arguments -- each returns a status
and leaves the context usable."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import dev, harmonic_case, host, plans, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def test_bounded_wait_times_out_and_context_survives(T):
    import torch
    T.ts_device_status()  # clear
    T.ts_selftest_wait_timeout(200_000_000)  # ~0.1 s at 2 GHz, then the kernel returns
    with pytest.raises(T.TsError) as e:
        T.ts_device_status()
    assert e.value.status == T.TS_ERR_TIMEOUT and "code 9" in str(e.value)
    T.ts_device_status()  # the flag was cleared by the previous read
    n = (32, 32, 32)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, 1 << 1)
    b = S.normal(2, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u, T.TS_BF16X3)
    torch.cuda.synchronize()
    assert rel(host(u), O.apply_inverse(Po, 0.5, b)) < 5e-5


def test_pcg_iteration_cap_returns_last_iterate(T):
    n = (24, 24, 24)
    L, f = harmonic_case(n, omega=(1, 1, 1))
    P, Po = plans(n, L, f)
    V2 = S.v2_cos_bumps(n, L, seed=1) + 5.0
    b = S.uniform(0, Po.N)
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 0.0, 0.0, dev(V2), dev(b), x, 1e-14, 2, allow_not_converged=True)
    assert st == T.TS_ERR_NOT_CONVERGED and it == 2
    xo, _, _ = O.pcg(Po, b, sigma=0.0, V2=V2, tol=1e-14, maxit=2)
    assert rel(host(x), xo) < 1e-10 and 0 < relres < 1.0


def test_non_finite_right_hand_side_is_reported(T):
    n = (16, 16, 16)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    b = S.uniform(0, Po.N)
    b[123] = math.nan
    x = dev(np.zeros(Po.N))
    st, it, relres = T.ts_pcg(P, 1.0, 1.0, None, dev(b), x, 1e-10, 10, allow_not_converged=True)
    assert st == T.TS_ERR_NOT_CONVERGED
    assert "non-finite" in T.ts_last_error() or not math.isfinite(relres)


def test_invalid_arguments_leave_the_library_usable(T):
    n = (16, 16)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f)
    b = dev(S.uniform(0, Po.N))
    with pytest.raises(T.TsError) as e:
        T.ts_apply_exp(P, 0.1, b, b, 7)
    assert e.value.status == T.TS_ERR_INVALID_ARG
    with pytest.raises(T.TsError) as e:
        T.ts_apply_inverse(P, 0.5, b, b, T.TS_BF16X3)   # precision not in the plan's mask
    assert e.value.status == T.TS_ERR_UNSUPPORTED
    with pytest.raises(T.TsError) as e:
        T.ts_split_step(P, 0.01, -1, b, b, T.TS_C128)
    assert e.value.status == T.TS_ERR_INVALID_ARG
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, b, u)
    assert rel(host(u), O.apply_inverse(Po, 0.5, host(b))) < 1e-12
