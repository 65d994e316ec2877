"""ts_apply_inverse_noalloc: the inverse apply for callers that must not allocate device
memory while they run (an application that owns the whole device through its own
allocator, or a latency-critical loop that cannot pay for cudaMalloc/cudaFree).  Its work
buffers live in a fixed 32 MiB array inside the library.

Checked through the C ABI against ts_apply_inverse on two calls in a row (the array keeps
the previous call's contents, so the second call must not depend on them), with the
tolerances of the other parity tests: 3D grids whose axes are multiples of 8, ragged
grids whose bf16 planes have padded rows (run right after an FP64 call has filled the
array with doubles, which read as arbitrary bf16 bit patterns), and 2D grids (an even
number of passes hands the FP64 buffers over in the other order).  Sizes above the fixed
limit and invalid precisions are refused with the statuses of ts_apply_inverse.  This
file is collected last on purpose."""
import numpy as np
import pytest

from paper_2605_20491_b300 import synth as S
from gpu_util import dev, harmonic_case, host, plans, rel

pytestmark = pytest.mark.gpu
MASK = (1 << 1) | (1 << 2)
MASK1 = MASK | (1 << 6)  # with TS_BF16X1


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


@pytest.mark.parametrize("prec,tol", [(1, 5e-5), (2, 1e-5), (6, 2e-2)])
@pytest.mark.parametrize("n", [(41, 23, 17), (57, 9, 33)])
def test_noalloc_ragged_planes_after_fp64_fill(T, n, prec, tol):
    """Axis lengths that are not multiples of 8: the bf16 planes of every pass have padded
    rows.  Before each split-precision call an FP64 call fills the whole region it uses
    with doubles; neither the padding nor anything else may be read from it."""
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK1)
    for call, seed in enumerate((31, 32)):
        junk = dev(1e300 * S.normal(seed + 10, P.N))
        T.ts_apply_inverse_noalloc(P, 0.5, junk, dev(np.zeros(P.N)), T.TS_FP64)
        b = dev(S.normal(seed, P.N))
        want = dev(np.zeros(P.N))
        T.ts_apply_inverse(P, 0.5, b, want, prec)
        got = dev(np.full(P.N, np.nan))
        T.ts_apply_inverse_noalloc(P, 0.5, b, got, prec)
        g, w = host(got), host(want)
        assert np.all(np.isfinite(g)), f"call {call}"
        assert rel(g, w) < tol, (call, rel(g, w))


@pytest.mark.parametrize("n", [(200, 136), (37, 64)])
def test_noalloc_two_dimensional_fp64(T, n):
    """d = 2: the FP64 passes end in the other work buffer than for odd d."""
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK)
    for call, seed in enumerate((41, 42)):
        b = dev(S.normal(seed, P.N))
        want = dev(np.zeros(P.N))
        T.ts_apply_inverse(P, 0.5, b, want, T.TS_FP64)
        got = dev(np.full(P.N, np.nan))
        T.ts_apply_inverse_noalloc(P, 0.5, b, got, T.TS_FP64)
        assert rel(host(got), host(want)) < 1e-12, call


def test_noalloc_precision_checks_match_apply_inverse(T):
    """An out-of-range precision is TS_ERR_INVALID_ARG and a precision outside the plan's
    mask is TS_ERR_UNSUPPORTED, for both entry points; the library stays usable."""
    n = (16, 16, 8)
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK)  # no TS_BF16X1
    x = dev(np.ones(P.N))
    y = dev(np.zeros(P.N))
    for prec, status in ((99, T.TS_ERR_INVALID_ARG), (-1, T.TS_ERR_INVALID_ARG), (6, T.TS_ERR_UNSUPPORTED)):
        for fn in (T.ts_apply_inverse, T.ts_apply_inverse_noalloc):
            with pytest.raises(T.TsError) as e:
                fn(P, 0.5, x, y, prec)
            assert e.value.status == status, (fn.__name__, prec)
    T.ts_apply_inverse_noalloc(P, 0.5, x, y, T.TS_BF16X3)
    want = dev(np.zeros(P.N))
    T.ts_apply_inverse(P, 0.5, x, want, T.TS_BF16X3)
    assert rel(host(y), host(want)) < 5e-5


def test_noalloc_limit_counts_padded_rows(T):
    """The size check uses the padded plane size: N = 4,177,665 is below the BF16X3 limit
    for grids whose axes are multiples of 8 (4,194,304), but the widest pass's planes
    (rows padded to 8 elements, 4,404,360 values) need 2 x 17.6 MB, above the 32 MiB."""
    n = (255, 129, 127)
    L, f = harmonic_case(n)
    P, _ = plans(n, L, f, MASK)
    x = dev(np.zeros(P.N))
    with pytest.raises(T.TsError) as e:
        T.ts_apply_inverse_noalloc(P, 1.0, x, x, T.TS_BF16X3)
    assert e.value.status == T.TS_ERR_INVALID_ARG and "multiple of 8" in str(e.value)
