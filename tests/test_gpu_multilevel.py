"""Multi-level shifted inverse iteration (Sec. 5.3.1) on the GPU: the tensor-product
linear interpolation between grids against the oracle, and Table multilevel's ground state
of the stirrer potential carried from 99^3 to 199^3 (Q^20)."""
import numpy as np
import pytest

from oracle import sem
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


PAIRS = [(((9, 14), 5, (2.0, 3.0)), ((39, 23), 2, (2.0, 3.0))),
         (((39, 19, 19), 20, (8.0, 8.0, 8.0)), ((79, 39, 59), 20, (8.0, 8.0, 8.0))),
         (((15, 7), 1, (1.0, 2.0)), ((59, 39), 20, (1.0, 2.0))),
         (((31,), 2, (4.0,)), ((17,), 3, (4.0,)))]


@pytest.mark.parametrize("coarse,fine", PAIRS)
def test_interpolation_vs_oracle(T, coarse, fine):
    """Element-wise; the tolerance covers the two sides' independently computed GLL nodes,
    which agree to ~1e-15 L: near the crowded ends of a Q^20 element (node gaps ~1e-3 L)
    that moves an interpolation fraction by ~1e-12 at most, times |u| <= 5."""
    (nc, kc, L), (nf, kf, _) = coarse, fine
    zc = [np.zeros(m) for m in nc]
    zf = [np.zeros(m) for m in nf]
    Pc, Pf = T.ts_plan_create(nc, L, zc, 0, order=kc), T.ts_plan_create(nf, L, zf, 0, order=kf)
    Oc, Of = sem.plan(nc, L, zc, kc), sem.plan(nf, L, zf, kf)
    uc = np.random.default_rng(1).standard_normal(Oc.N)
    uf = dev(np.zeros(Of.N))
    T.ts_interpolate(Pc, dev(uc), Pf, uf)
    np.testing.assert_allclose(host(uf), sem.interpolate(Oc, uc, Of), rtol=0, atol=5e-12)


def _stirrer_level(T, n):
    import torch
    k, L = 20, 8.0
    x, _ = T.ts_grid_nodes(n, L, k)
    P = T.ts_plan_create((n,) * 3, (L,) * 3, [x ** 2, x ** 2, 4 * x ** 2], 1 << T.TS_BF16X3, order=k)
    xs = torch.from_numpy(x).cuda()
    V2 = (8.0 * torch.exp(-((xs[None, None, :] - 1.0) ** 2 + xs[None, :, None] ** 2))).expand(n, n, n)
    return P, V2.contiguous().reshape(-1)


def test_paper_multilevel_stirrer(T):
    """Table multilevel: H = -Delta + x^2 + y^2 + 4 z^2 + 8 exp(-((x - 1)^2 + y^2)) on [-8, 8]^3,
    Q^20, shift 0.9 lambda_min(A), PCG tolerance 1e-12, |d lambda| / |lambda| < 1e-13;
    inverse iteration at 99^3 from the ground state of A, then at 199^3 from its
    interpolated eigenvector: lambda_1 = 5.286155366963, and the finer level needs far
    fewer outer iterations than the coarse one (table: 30, then 21 at 199^3)."""
    import torch
    levels = [_stirrer_level(T, 99), _stirrer_level(T, 199)]
    plans = [p for p, _ in levels]
    lam_min = sum(T.ts_plan_eigs(plans[0], a)[0] for a in range(3))
    u = torch.empty(plans[-1].N, dtype=torch.float64, device="cuda")
    lam, outer, pcg = T.ts_inverse_iteration_multilevel(plans, [v for _, v in levels], 0.9 * lam_min, u, 1e-13, 200,
                                                        1e-12, 500, T.TS_BF16X3)
    print(f"multilevel: lambda {lam!r}, outer {outer}, pcg {pcg}")
    assert abs(lam - 5.286155366963) < 1e-12
    assert outer[1] < outer[0]


def _coulomb_level(T, n, delta):
    import torch
    k, L = 10, 8.0
    x, _ = T.ts_grid_nodes(n, L, k)
    P = T.ts_plan_create((n,) * 4, (L,) * 4, [x ** 2] * 4, 1 << T.TS_BF16X3, order=k)
    xs = torch.from_numpy(x).cuda()
    # axes 1, 2: particle 1 (x_1a, x_1b); axes 3, 4: particle 2; vec order, axis 1 fastest
    d2 = (xs[None, :, None, None] - xs[:, None, None, None]) ** 2 + (xs[None, None, None, :] - xs[None, None, :, None]) ** 2
    V2 = 1.0 / torch.sqrt(d2 + delta * delta)  # c = 1
    return P, V2.reshape(-1).contiguous()


def test_paper_pcg_precond_iterations(T):
    """Table pcg_precond: PCG on (-Delta + V1 + V2) u = f, the 4D Coulomb system with
    delta = 0.01 on 49^4 Q^10, random f, tolerance 1e-12, FP64, preconditioner
    (-Delta + V1)^{-1}: 24 iterations (the comparison preconditioners are other methods)."""
    import torch
    P, V2 = _coulomb_level(T, 49, 0.01)
    f = torch.from_numpy(np.random.default_rng(7).standard_normal(P.N)).cuda()
    x = torch.zeros_like(f)
    _, it, relres = T.ts_pcg(P, 0.0, 0.0, V2, f, x, 1e-12, 500, T.TS_FP64)
    print(f"pcg_precond: {it} iterations, relres {relres:.2e}")
    assert relres < 1e-11 and abs(it - 24) <= 3
