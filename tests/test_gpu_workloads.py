"""Full-size workloads on the GPU, checked through the oracle where it can still run (the
FP64 stencil over all points) and through properties that hold at any size."""
import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def test_n512_refined_solve_full_size(T):
    """The benchmark's solve at n = 512 (1.34e8 DoF), in the benchmark's configuration:
    the oracle's FP64 stencil residual ||b - A u|| / ||b|| of the GPU solution (computed on
    the host over every grid point) and agreement with the FP64 GPU apply."""
    import torch
    w = S.WORKLOADS["3d_n512_apply"]
    n, L = w["n"], w["L"]
    f = S.harmonic(n, L, w["omega"])
    P = T.ts_plan_create(n, L, f, 1 << T.TS_BF16X3)
    b_h = S.normal(w["seed"], P.N)
    b = torch.from_numpy(b_h).cuda()
    u = torch.empty_like(b)
    T.ts_solve_refined(P, w["sigma"], b, u, T.TS_BF16X3, 2)
    u64 = torch.empty_like(b)
    T.ts_apply_inverse(P, w["sigma"], b, u64, T.TS_FP64)
    assert ((u - u64).norm() / u64.norm()).item() < 1e-12
    Po = O.Plan(tuple(n), tuple(L), f)
    uh = host(u)
    r = O.stencil(Po, uh, w["sigma"]) - b_h
    assert np.linalg.norm(r) / np.linalg.norm(b_h) < 1e-11


def test_n256_inverse_iteration_full_size(T):
    """The 3D PCG workload (n = 256, V2 = 5 cos cos cos + 8 bumps): shifted inverse iteration
    with the BF16X3 preconditioner agrees with the FP64-preconditioned run on lambda, and
    the eigen-residual ||H u - lambda u|| is small."""
    import torch
    w = S.WORKLOADS["3d_n256_pcg"]
    n, L = w["n"], w["L"]
    f = S.harmonic(n, L, w["omega"])
    P = T.ts_plan_create(n, L, f, 1 << T.TS_BF16X3)
    V2h = S.v2_cos_bumps(n, L, seed=w["v2_seed"])
    V2 = torch.from_numpy(V2h).cuda()
    shift = sum(T.ts_plan_eigs(P, k)[0] for k in range(3)) + V2h.min() - 1.0
    res = {}
    for prec in (T.TS_BF16X3, T.TS_FP64):
        u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
        lam, outer, pcg = T.ts_inverse_iteration(P, shift, V2, u, True, 1e-12, 400, 1e-10, 500, prec)
        res[prec] = (lam, outer, pcg, u)
    l1, l2 = res[T.TS_BF16X3][0], res[T.TS_FP64][0]
    assert abs(l1 - l2) / abs(l2) < 1e-10
    u = res[T.TS_BF16X3][3]
    Hu = torch.empty_like(u)
    T.ts_apply_operator(P, 0.0, V2, u, Hu)
    assert ((Hu - l1 * u).norm() / abs(l1)).item() < 1e-5
    assert (u.sum() > 0).item()
    # Weyl: lambda_min(A) + min V2 <= lambda_1 <= lambda_min(A) + max V2
    lamA = sum(T.ts_plan_eigs(P, k)[0] for k in range(3))
    assert lamA + V2h.min() <= l1 <= lamA + V2h.max()
    # the oracle's own FP64 operator (eq. general_system, plain loops over every point) on the
    # GPU eigenvector: its Rayleigh quotient equals the GPU lambda and its eigen-residual is small
    Po = O.Plan(tuple(n), tuple(L), f)
    uh = host(u)
    Hu_o = O.stencil(Po, uh, 0.0, V2h)
    lam_o = float(uh @ Hu_o / (uh @ uh))
    assert abs(lam_o - l1) / abs(l1) < 1e-11, (lam_o, l1)
    assert np.linalg.norm(Hu_o - lam_o * uh) / (abs(lam_o) * np.linalg.norm(uh)) < 1e-5
