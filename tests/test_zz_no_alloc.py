"""ts_apply_inverse_noalloc: the inverse apply for callers that must not allocate device
memory while they run (an application that owns the whole device through its own
allocator, or a latency-critical loop that cannot pay for cudaMalloc/cudaFree).  Its work
buffers live in a fixed 32 MiB array inside the library.

Checked through the C ABI against ts_apply_inverse on two calls in a row (the array keeps
the previous call's contents, so the second call must not depend on them), with the
tolerances of the other parity tests; sizes above the fixed limit are refused.  This file
is collected last on purpose."""
import numpy as np
import pytest

from paper_2605_20491_b300 import synth as S
from gpu_util import dev, harmonic_case, host, plans, rel

pytestmark = pytest.mark.gpu
MASK = (1 << 1) | (1 << 2)


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 5e-5), (2, 1e-5)])
@pytest.mark.parametrize("n", [(64, 48, 40), (128, 128, 128)])
def test_noalloc_matches_apply_inverse_twice(T, n, prec, tol):
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK)
    if prec == 2 and P.N * 12 > (32 << 20):
        pytest.skip("above the BF16X6 limit of the fixed scratch")
    for call, seed in enumerate((21, 22)):
        b = dev(S.normal(seed, P.N))
        want = dev(np.zeros(P.N))
        T.ts_apply_inverse(P, 0.5, b, want, prec)
        got = dev(np.full(P.N, np.nan))
        T.ts_apply_inverse_noalloc(P, 0.5, b, got, prec)
        g, w = host(got), host(want)
        assert np.all(np.isfinite(g)), f"call {call}"
        assert rel(g, w) < tol, (call, rel(g, w))


def test_noalloc_in_place_and_limit(T):
    n = (40, 24, 16)
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK)
    b = dev(S.normal(3, P.N))
    want = dev(np.zeros(P.N))
    T.ts_apply_inverse(P, 1.0, b, want, T.TS_BF16X3)
    T.ts_apply_inverse_noalloc(P, 1.0, b, b, T.TS_BF16X3)  # b and u alias
    assert rel(host(b), host(want)) < 5e-5
    big = (256, 128, 128)  # 4,194,304 DoF: fits BF16X3 exactly, not FP64
    Lb, fb = harmonic_case(big)
    Pb, _ = plans(big, Lb, fb, MASK)
    x = dev(np.zeros(Pb.N))
    with pytest.raises(T.TsError) as e:
        T.ts_apply_inverse_noalloc(Pb, 1.0, x, x, T.TS_FP64)
    assert e.value.status == T.TS_ERR_INVALID_ARG and "DoF" in str(e.value)
    T.ts_apply_inverse_noalloc(Pb, 1.0, x, x, T.TS_BF16X3)
