"""Parity of the split-precision (tcgen05) path with the CPU oracle, through the C ABI.

Shapes cover a ragged M tail (R not a multiple of 128), K tails (n not a multiple of 64),
N tails (n > 256 and not a multiple of the N tile) and several tiles per pass.

Tolerances (relative l2 against the FP64 oracle), from the arithmetic: a 2-term bf16
split carries 16 bits (unit 2^-17 per value and per table entry), so each pass adds
O(2^-16) relative error; 2d passes stay below 5e-5 (BF16X3, measured about 1e-5).  A
3-term split carries 24 bits, so the FP32 accumulation inside the tensor core
(O(sqrt(n) 2^-24) per pass) dominates: below 1e-5 for 2d passes (BF16X6, measured
2e-6 to 4e-6).  Complex64 output adds one FP32 rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import MAXNORM_FACTOR, dev, harmonic_case, host, maxrel, plans, rel

pytestmark = pytest.mark.gpu
TOL = {1: 5e-5, 2: 1e-5}   # TS_BF16X3, TS_BF16X6
MASK = (1 << 1) | (1 << 2)

SHAPES = [(64, 64, 64), (40, 24, 8), (128, 96, 40), (264, 16), (8, 8, 8, 8, 8), (32, 32, 32)]


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", SHAPES)
def test_inverse_mixed_vs_oracle(T, n, prec):
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    b = S.normal(2, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u, prec)
    T.ts_device_status()
    want = O.apply_inverse(Po, 0.5, b)
    err = rel(host(u), want)
    assert err < TOL[prec], err
    assert maxrel(host(u), want) < MAXNORM_FACTOR * TOL[prec]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", [(64, 48, 32), (40, 24, 8), (16, 16, 16, 16), (272, 8)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_exp_mixed_vs_oracle(T, n, prec, dtype):
    L, f = harmonic_case(n, L=4.0)
    P, Po = plans(n, L, f, MASK)
    psi = S.complex_normal(3, Po.N)
    if dtype == "c128":
        out = dev(np.zeros(2 * Po.N))
        T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C128, prec)
        tol = TOL[prec]
    else:
        psi = psi.astype(np.float32)
        out = dev(np.zeros(2 * Po.N, dtype=np.float32))
        T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C64, prec)
        tol = max(TOL[prec], 1e-6)
    T.ts_device_status()
    got = host(out).astype(np.float64)
    want = O.apply_exp(Po, 0.01, psi.astype(np.float64))
    err = rel(got, want)
    assert err < tol, err
    assert maxrel(got, want) < MAXNORM_FACTOR * tol


def test_mixed_rejects_unsupported(T):
    n = (12, 16)
    L, f = harmonic_case(n)
    b = dev(np.ones(12 * 16))
    P2, _ = plans((16, 16), L, [f[1], f[1]], 0)
    with pytest.raises(T.TsError) as e:
        T.ts_apply_inverse(P2, 1.0, b[:256], b[:256], T.TS_BF16X3)
    assert e.value.status == T.TS_ERR_UNSUPPORTED


@pytest.mark.parametrize("n", [(64, 64, 64), (128, 96, 40), (40, 24, 8), (16, 16, 16, 16)])
def test_refined_solve_reaches_fp64_accuracy(T, n):
    """Two refinements of the BF16X3 inverse reach FP64 rounding (< 1e-12 vs the oracle);
    zero refinements is the single split-precision apply."""
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    b = S.normal(2, Po.N)
    want = O.apply_inverse(Po, 0.5, b)
    bt = dev(b)
    errs = []
    for k in (0, 1, 2):
        u = dev(np.zeros(Po.N))
        T.ts_solve_refined(P, 0.5, bt, u, T.TS_BF16X3, k)
        errs.append(rel(host(u), want))
    assert errs[0] < TOL[1]
    assert errs[1] < 1e-8
    assert errs[2] < 1e-12, errs
    u1 = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, bt, u1, T.TS_BF16X3)
    u0 = dev(np.zeros(Po.N))
    T.ts_solve_refined(P, 0.5, bt, u0, T.TS_BF16X3, 0)
    assert np.array_equal(host(u0), host(u1))


@pytest.mark.parametrize("n", [(40, 24, 56), (72, 40, 40), (24, 40), (16, 8, 24, 32)])
def test_refined_solve_isotropic_ragged(T, n):
    """Equal spacing h = 1/2 on axes of unequal, ragged lengths (the residual's fixed-point
    Laplacian: tile edges along every axis, d = 2, 3, 4) reaches FP64 accuracy."""
    L = tuple((k + 1) / 4.0 for k in n)
    f = S.harmonic(n, L, tuple(1.0 + 0.2 * k for k in range(len(n))))
    P, Po = plans(n, L, f, MASK)
    b = S.normal(6, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_solve_refined(P, 0.25, dev(b), u, T.TS_BF16X3, 2)
    assert rel(host(u), O.apply_inverse(Po, 0.25, b)) < 1e-12


@pytest.mark.parametrize("n", [(64, 64, 64), (48, 40, 32)])
def test_refined_solve_zero_rhs_and_power_of_two_scaling(T, n):
    """b = 0 gives u = 0 exactly.  Every step of the refined solve commutes with scaling by a
    power of two (bf16 splits, FP32 products and tables, the residual's global fixed-point
    exponent), so u(2^k b) equals 2^k u(b) bit for bit on isotropic and anisotropic grids."""
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    u = dev(np.full(Po.N, 3.0))
    T.ts_solve_refined(P, 0.5, dev(np.zeros(Po.N)), u, T.TS_BF16X3, 2)
    assert not host(u).any()
    b = S.normal(5, Po.N) * (1.0 + 1e3 * (np.arange(Po.N) % 7 == 0))
    ref = dev(np.zeros(Po.N))
    T.ts_solve_refined(P, 0.5, dev(b), ref, T.TS_BF16X3, 2)
    ref = host(ref)
    assert rel(ref, O.apply_inverse(Po, 0.5, b)) < 1e-12
    for k in (-20, 37):
        uk = dev(np.zeros(Po.N))
        T.ts_solve_refined(P, 0.5, dev(np.ldexp(b, k)), uk, T.TS_BF16X3, 2)
        assert np.array_equal(host(uk), np.ldexp(ref, k))


def test_autotune_cache_roundtrip(T, tmp_path):
    """The autotuner searches each axis length once, writes the cache, and a second call
    applies the cached choice without timing; results stay within tolerance."""
    n = (64, 48, 64)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    cache = str(tmp_path / "tune.txt")
    assert T.ts_autotune(P, T.TS_R64, T.TS_BF16X3, cache) == 2
    lines = open(cache).read().split("\n")
    assert len([x for x in lines if x.strip()]) == 2
    assert T.ts_autotune(P, T.TS_R64, T.TS_BF16X3, cache) == 0
    b = S.normal(2, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u, T.TS_BF16X3)
    assert rel(host(u), O.apply_inverse(Po, 0.5, b)) < TOL[1]
    T.ts_tc_config_reset(False, 64)
    T.ts_tc_config_reset(False, 48)


PAIR_SHAPES = [(64, 64, 64), (40, 24, 8), (264, 16), (128, 96, 48), (512, 24)]


# N-tile caps (real, complex): the narrower pair first (256 TMEM columns per CTA), then the
# full-width tiles (all 512 columns).
@pytest.mark.parametrize("n,caps", [(n, (128, 64)) for n in PAIR_SHAPES] + [(n, (256, 128)) for n in PAIR_SHAPES])
def test_cta_pairs_match_single_cta(T, n, caps):
    """CTA pairs sharing each tensor-core instruction (256-row units, each CTA staging half
    of the S_k tile; ragged M tails leave the second CTA of the last pair with rows beyond
    the tensor) give bit-identical results to single-CTA passes, which accumulate the same
    products in the same K order, for BF16X3 inverse applies and BF16X6 complex exponentials."""
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    b = dev(S.normal(2, Po.N))
    psi = dev(S.complex_normal(3, Po.N))

    def run(cluster):
        try:
            T.ts_tc_config_set(False, 0, 64, caps[0], cluster)
            T.ts_tc_config_set(True, 0, 64, caps[1], cluster)
            u = dev(np.zeros(Po.N))
            T.ts_apply_inverse(P, 0.5, b, u, T.TS_BF16X3)
            out = dev(np.zeros(2 * Po.N))
            T.ts_apply_exp(P, 0.01, psi, out, T.TS_C128, T.TS_BF16X6)
            T.ts_device_status()
        finally:
            T.ts_tc_config_reset(False)
            T.ts_tc_config_reset(True)
        return host(u), host(out)

    u_pair, out_pair = run(T.TS_TC_PAIR)
    u_one, out_one = run(1)
    assert rel(u_pair, O.apply_inverse(Po, 0.5, host(b))) < TOL[1]
    assert rel(out_pair, O.apply_exp(Po, 0.01, host(psi))) < TOL[2]
    assert np.array_equal(u_pair, u_one)
    assert np.array_equal(out_pair, out_one)


MASK1 = MASK | (1 << 6)  # TS_BF16X1


@pytest.mark.parametrize("n", [(64, 64, 64), (40, 24, 8), (128, 96, 48)])
def test_bf16x1_apply_is_coarse_inverse(T, n):
    """One bf16 plane and one product per contraction: the inverse and the complex
    exponential agree with the oracle to the bf16 rounding of the data and of S_k
    accumulated over 2d passes (a few 1e-3 relative)."""
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK1)
    b = S.normal(2, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u, T.TS_BF16X1)
    e_inv = rel(host(u), O.apply_inverse(Po, 0.5, b))
    psi = S.complex_normal(3, Po.N)
    out = dev(np.zeros(2 * Po.N))
    T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C128, T.TS_BF16X1)
    e_exp = rel(host(out), O.apply_exp(Po, 0.01, psi))
    T.ts_device_status()
    assert 1e-4 < e_inv < 2e-2, e_inv
    assert 1e-4 < e_exp < 2e-2, e_exp


@pytest.mark.parametrize("n", [(64, 64, 64), (128, 96, 48), (40, 24, 8)])
def test_schedule_reaches_target(T, n):
    """A precision per apply: BF16X3, a BF16X3 refinement and a BF16X1 refinement end below
    1e-10 (the error contracts by each apply's relative error); BF16X1 alone needs about
    six applies for the same; the all-BF16X3 schedule equals ts_solve_refined bit for bit."""
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK1)
    b = S.normal(2, Po.N)
    want = O.apply_inverse(Po, 0.5, b)
    bt = dev(b)
    X1, X3 = T.TS_BF16X1, T.TS_BF16X3
    errs = {}
    for name, sched in {"331": [X3, X3, X1], "1x6": [X1] * 6, "33": [X3, X3], "333": [X3, X3, X3]}.items():
        u = dev(np.zeros(Po.N))
        T.ts_solve_schedule(P, 0.5, bt, u, sched)
        errs[name] = rel(host(u), want)
        if name == "333":
            ur = dev(np.zeros(Po.N))
            T.ts_solve_refined(P, 0.5, bt, ur, X3, 2)
            assert np.array_equal(host(u), host(ur))
    assert errs["331"] < 1e-10, errs
    assert errs["1x6"] < 1e-9, errs
    assert errs["331"] < errs["33"], errs


def test_schedule_rejects_bad_entries(T):
    n = (16, 16, 16)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)  # BF16X1 not in the mask
    b = dev(np.ones(Po.N))
    u = dev(np.zeros(Po.N))
    for sched in ([], [T.TS_FP64], [T.TS_BF16X3, T.TS_FP32], [T.TS_BF16X3, T.TS_BF16X1], [T.TS_BF16X3] * 18):
        with pytest.raises(T.TsError) as e:
            T.ts_solve_schedule(P, 0.5, b, u, sched)
        assert e.value.status in (T.TS_ERR_INVALID_ARG, T.TS_ERR_UNSUPPORTED)
    T.ts_solve_schedule(P, 0.5, b, u, [T.TS_BF16X3, T.TS_BF16X6])


BATCH_CASES = [((32, 48, 64), "inv", 1), ((64, 64, 64), "inv", 1), ((40, 24, 8), "c128", 1), ((96, 32, 48), "c64", 6),
               ((16, 16, 16, 16), "inv", 2), ((264, 16), "inv", 1), ((256, 16, 16), "inv", 1), ((48, 48, 48), "c128", 2),
               ((24, 40, 56), "inv", 6)]


def test_apply_batch_equals_single_calls(T):
    """ts_apply_batch runs every stage of all items in one launch per (precision, data kind)
    group (work-list tensor-core passes over heterogeneous grids: d = 2, 3, 4, ragged n,
    real and complex, BF16X1/X3/X6); each item's result equals its own single call bit for
    bit, and one of them matches the oracle."""
    import torch
    items, singles = [], []
    for q, (n, kind, prec) in enumerate(BATCH_CASES):
        L, f = harmonic_case(n)
        P, Po = plans(n, L, f, MASK1)
        if kind == "inv":
            x = dev(S.normal(10 + q, Po.N))
            out = dev(np.zeros(Po.N))
            ref = dev(np.zeros(Po.N))
            T.ts_apply_inverse(P, 0.5, x, ref, prec)
            items.append((P, T.TS_R64, prec, 0.5, x, out))
        else:
            dt = T.TS_C128 if kind == "c128" else T.TS_C64
            z = S.complex_normal(10 + q, Po.N)
            x = dev(z) if kind == "c128" else dev(z.astype(np.float32))
            out = torch.zeros_like(x)
            ref = torch.zeros_like(x)
            T.ts_apply_exp(P, 0.01, x, ref, dt, prec)
            items.append((P, dt, prec, 0.01, x, out))
        singles.append((ref, Po, kind))
    T.ts_apply_batch(items)
    T.ts_device_status()
    for (P, dt, prec, param, x, out), (ref, Po, kind) in zip(items, singles):
        assert np.array_equal(host(out), host(ref)), (Po.n, kind, prec)
    P, dt, prec, param, x, out = items[1]
    assert rel(host(out), O.apply_inverse(singles[1][1], 0.5, host(x))) < TOL[1]
    T.ts_apply_batch([])


def test_apply_batch_rejects_bad_items(T):
    n = (16, 16, 16)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    x = dev(np.ones(Po.N))
    y = dev(np.zeros(Po.N))
    for bad in [(P, T.TS_R64, T.TS_FP64, 0.5, x, y), (P, T.TS_R64, T.TS_BF16X1, 0.5, x, y), (P, 7, T.TS_BF16X3, 0.5, x, y)]:
        with pytest.raises(T.TsError):
            T.ts_apply_batch([(P, T.TS_R64, T.TS_BF16X3, 0.5, x, y), bad])


# Any n: the planes and tables store each pass's contracted axis in rows padded to a
# multiple of 8 (16-byte TMA rows); the writers of every plane (input split, pass
# epilogues, the three residual kernels) and the final unpadded FP64 / complex stores.
RAGGED = [(12, 16), (33, 9, 21), (99,), (5, 7, 3, 9), (100, 37, 51), (1, 17, 3), (129, 65)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", RAGGED)
def test_inverse_any_n_vs_oracle(T, n, prec):
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    b = S.normal(2, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u, prec)
    T.ts_device_status()
    assert rel(host(u), O.apply_inverse(Po, 0.5, b)) < TOL[prec]


@pytest.mark.parametrize("n", [(33, 9, 21), (5, 7, 3, 9), (99,)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_exp_any_n_vs_oracle(T, n, dtype):
    L, f = harmonic_case(n, L=4.0)
    P, Po = plans(n, L, f, MASK)
    psi = S.complex_normal(3, Po.N)
    if dtype == "c128":
        out = dev(np.zeros(2 * Po.N))
        T.ts_apply_exp(P, 0.01, dev(psi), out, T.TS_C128, T.TS_BF16X3)
    else:
        out = dev(np.zeros(2 * Po.N, dtype=np.float32))
        T.ts_apply_exp(P, 0.01, dev(psi.astype(np.float32)), out, T.TS_C64, T.TS_BF16X3)
    T.ts_device_status()
    got = host(out).astype(np.float64)
    assert rel(got, O.apply_exp(Po, 0.01, psi).view(np.float64)) < max(TOL[1], 1e-6)


@pytest.mark.parametrize("n,iso", [((33, 33, 33), True), ((41, 19, 27), True), ((33, 9, 21), False),
                                   ((5, 7, 3, 9), False), ((99, 45), True)])
def test_refined_any_n_reaches_fp64(T, n, iso):
    """Refinements with residuals split into padded planes: the exact fixed-point kernels
    (equal spacing; d = 3 uses the marching form) and the FP64 stencil (unequal spacing)."""
    L = tuple((k + 1) / 4.0 for k in n) if iso else tuple(1.0 + 0.5 * a for a in range(len(n)))
    f = S.harmonic(n, L, tuple(1.0 + 0.2 * k for k in range(len(n))))
    P, Po = plans(n, L, f, MASK | (1 << 6))
    b = S.normal(6, Po.N)
    want = O.apply_inverse(Po, 0.25, b)
    u = dev(np.zeros(Po.N))
    T.ts_solve_refined(P, 0.25, dev(b), u, T.TS_BF16X3, 2)
    assert rel(host(u), want) < 1e-12
    T.ts_solve_schedule(P, 0.25, dev(b), u, [T.TS_BF16X3, T.TS_BF16X3, T.TS_BF16X1])
    assert rel(host(u), want) < 1e-10


def test_apply_batch_any_n(T):
    """Work-list passes over grids of unrelated ragged shapes equal their single calls."""
    import torch
    cases = [((33, 9, 21), "inv", T.TS_BF16X3), ((5, 7, 3, 9), "c128", T.TS_BF16X3), ((99,), "inv", T.TS_BF16X6),
             ((12, 16), "c64", T.TS_BF16X3), ((40, 24, 8), "inv", T.TS_BF16X3)]
    items, refs = [], []
    for q, (n, kind, prec) in enumerate(cases):
        L, f = harmonic_case(n)
        P, Po = plans(n, L, f, MASK)
        if kind == "inv":
            x = dev(S.normal(20 + q, Po.N))
            out, ref = dev(np.zeros(Po.N)), dev(np.zeros(Po.N))
            T.ts_apply_inverse(P, 0.5, x, ref, prec)
            items.append((P, T.TS_R64, prec, 0.5, x, out))
        else:
            dt = T.TS_C128 if kind == "c128" else T.TS_C64
            z = S.complex_normal(20 + q, Po.N)  # interleaved (re, im)
            x = dev(z) if kind == "c128" else dev(z.astype(np.float32))
            out, ref = torch.zeros_like(x), torch.zeros_like(x)
            T.ts_apply_exp(P, 0.01, x, ref, dt, prec)
            items.append((P, dt, prec, 0.01, x, out))
        refs.append(ref)
    T.ts_apply_batch(items)
    T.ts_device_status()
    for it, ref in zip(items, refs):
        assert np.array_equal(host(it[5]), host(ref))


def test_noalloc_any_n(T):
    n = (33, 9, 21)
    L, f = harmonic_case(n)
    P, Po = plans(n, L, f, MASK)
    b = S.normal(7, Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse_noalloc(P, 0.5, dev(b), u, T.TS_BF16X3)
    u2 = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.5, dev(b), u2, T.TS_BF16X3)
    assert np.array_equal(host(u), host(u2))
    assert rel(host(u), O.apply_inverse(Po, 0.5, b)) < TOL[1]


@pytest.mark.parametrize("n,offset", [((64, 48, 40), 0), ((40, 72, 24), 0), ((63, 64, 40), 0), ((64, 48, 40), 1)])
def test_refined_solve_fixed_point_iterate(T, n, offset):
    """On grids with one spacing and an even axis-0 length the refined solve keeps its
    iterate in 64-bit fixed point (U_0 stored, corrections added in integer arithmetic,
    residuals read U); an odd axis-0 length or a right-hand side not 16-byte aligned takes
    the FP64 iterate.  Both reach FP64 accuracy against the oracle, for the benchmark's
    schedule (BF16X3, BF16X3, BF16X1), two BF16X3 refinements and a single refinement."""
    import torch
    L = tuple((k + 1) / 4.0 for k in n)
    f = S.harmonic(n, L, (1.0, 1.3, 0.7))
    P, Po = plans(n, L, f, MASK | (1 << 6))
    b = S.normal(9, Po.N)
    want = O.apply_inverse(Po, 0.5, b)
    storage = dev(np.concatenate([np.zeros(offset), b]))
    bt = storage[offset:]
    for sched, tol in (([1, 1, 6], 1e-11), ([1, 1, 1], 1e-12), ([1, 1], 5e-9)):
        u = dev(np.full(Po.N, np.nan))
        T.ts_solve_schedule(P, 0.5, bt, u, sched)
        T.ts_device_status()
        assert rel(host(u), want) < tol, (sched, rel(host(u), want))
    # b = 0 gives u = 0 exactly on both forms
    u = dev(np.full(Po.N, 3.0))
    T.ts_solve_schedule(P, 0.5, torch.zeros_like(bt), u, [1, 1, 6])
    assert not host(u).any()
