"""Hermite spectral plans (order -1, Appendix app:hermite) on the GPU: FP64 parity with the
oracle (oracle/hermite.py), PCG against the oracle's operator, Table hermite_accuracy at
all three printed sizes, and one entry of Table magnus2_hermite at the table's 499^3."""
import math

import numpy as np
import pytest

from oracle import hermite as H
from oracle import sem
from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def _case(T, n):
    f = [(0.5 + 0.2 * a) * H.golub_welsch_nodes(n[a]) ** 2 for a in range(len(n))]
    P = T.ts_plan_create(n, (1.0,) * len(n), f, 0, order=-1)
    return P, H.plan(n, f), f


@pytest.mark.parametrize("n", [(24, 31, 17), (64,), (40, 33)])
def test_inverse_and_exp_fp64_vs_oracle(T, n):
    P, Po, _ = _case(T, n)
    rng = np.random.default_rng(0)
    # smooth, decaying data (products of Gaussians times low polynomials), as the basis represents
    X = [H.golub_welsch_nodes(m) for m in n]
    b = np.ones(())
    for a in range(len(n)):
        sh = [1] * len(n)
        sh[len(n) - 1 - a] = n[a]
        b = b * ((1.0 + 0.3 * X[a] + rng.uniform(-0.2, 0.2) * X[a] ** 2) * np.exp(-0.5 * X[a] ** 2)).reshape(sh)
    b = b.reshape(-1)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.7, dev(b), u)
    assert rel(host(u), H.apply_inverse(Po, 0.7, b)) < 1e-11
    psi = b * (1.0 + 0.5j)
    out = dev(np.zeros(2 * Po.N))
    T.ts_apply_exp(P, 0.05, dev(psi.view(np.float64)), out, T.TS_C128)
    assert rel(host(out).view(np.complex128), H.apply_exp(Po, 0.05, psi)) < 1e-11


def test_pcg_on_hermite_grid(T):
    """PCG with P = (-Delta + V1)^{-1} on R^2 (the appendix's Figure pcg_hermite setting, with
    a bounded V2): the solution satisfies (-D^2 x I + I x -D^2 + V1 + V2) x = b with -D^2 from
    the oracle, and V2 = 0 reproduces the direct solve."""
    n = (40, 33)
    P, Po, f = _case(T, n)
    X = [H.golub_welsch_nodes(m) for m in n]
    V2 = (2.0 * np.exp(-((X[0][None, :] - 1.0) ** 2 + X[1][:, None] ** 2))).reshape(-1)
    b = (np.exp(-0.5 * X[0] ** 2)[None, :] * (1 + X[1][:, None]) * np.exp(-0.5 * X[1] ** 2)[:, None]).reshape(-1)
    x = dev(np.zeros(Po.N))
    _, it, relres = T.ts_pcg(P, 0.0, 0.0, dev(V2), dev(b), x, 1e-11, 100)
    K = [H.axis_1d(m).K0 for m in n]
    xs = host(x).reshape(n[1], n[0])
    Ax = xs @ K[0].T + K[1] @ xs + (f[0][None, :] + f[1][:, None] + V2.reshape(n[1], n[0])) * xs
    assert np.linalg.norm(Ax.reshape(-1) - b) < 1e-8 * np.linalg.norm(b)
    assert it < 20
    x0 = dev(np.zeros(Po.N))
    _, it0, _ = T.ts_pcg(P, 0.0, 0.0, None, dev(b), x0, 1e-12, 100)
    assert it0 <= 2 and rel(host(x0), H.apply_inverse(Po, 0.0, b)) < 1e-10


def test_hermite_split_precision_and_interpolation_guard(T):
    """The tensor-core split-precision inverse works on Hermite grids too (the folded
    operands W^{+-1/2} Q stay moderate); interpolation, defined between bounded boxes, is
    refused."""
    n = (24, 16, 40)
    f = [(0.5 + 0.2 * a) * H.golub_welsch_nodes(n[a]) ** 2 for a in range(3)]
    P = T.ts_plan_create(n, (1.0,) * 3, f, 1 << T.TS_BF16X3, order=-1)
    Po = H.plan(n, f)
    b = np.random.default_rng(2).standard_normal(Po.N)
    u = dev(np.zeros(Po.N))
    T.ts_apply_inverse(P, 0.7, dev(b), u, T.TS_BF16X3)
    assert rel(host(u), H.apply_inverse(Po, 0.7, b)) < 5e-5
    with pytest.raises(T.TsError) as e:
        T.ts_interpolate(P, u, P, dev(np.zeros(Po.N)))
    assert e.value.status == T.TS_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,rel_printed,w_printed", [(199, 6.31e-5, 1.53e-5), (399, 2.20e-5, 4.05e-6),
                                                     (599, 1.20e-5, 1.87e-6)])
def test_paper_table_hermite_accuracy(T, n, rel_printed, w_printed):
    """Table hermite_accuracy (FP64): -Delta + V, V of eq. test_potential, on R^3;
    u* = prod_k sin(k pi (x_k + 1) / 2) / (1 + x_k^2); l2 relative error and Gauss-Hermite
    weighted L2 error, each to its three printed digits."""
    import torch
    x, _ = T.ts_grid_nodes(n, 1.0, -1)
    f = [1600 * np.sin(np.pi * x / 4) ** 2 + (a + 1) * x ** 2 for a in range(3)]
    P = T.ts_plan_create((n,) * 3, (1.0,) * 3, f, 0, order=-1)
    xs = torch.from_numpy(x).cuda()

    def factor(kk):
        s, c, g = torch.sin(kk * (xs + 1)), torch.cos(kk * (xs + 1)), 1.0 / (1.0 + xs ** 2)
        return s * g, -kk ** 2 * s * g + 2 * kk * c * (-2 * xs * g ** 2) + s * (6 * xs ** 2 - 2) * g ** 3

    (ux, dx), (uy, dy), (uz, dz) = factor(math.pi / 2), factor(math.pi), factor(1.5 * math.pi)
    fz, fy, fx = (torch.from_numpy(v).cuda() for v in (f[2], f[1], f[0]))
    U = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    b = (fz[:, None, None] + fy[None, :, None] + fx[None, None, :]) * U
    b -= dz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    b -= uz[:, None, None] * dy[None, :, None] * ux[None, None, :]
    b -= uz[:, None, None] * uy[None, :, None] * dx[None, None, :]
    u = torch.empty_like(b)
    T.ts_apply_inverse(P, 0.0, b.reshape(-1), u.reshape(-1))
    u -= U
    err = (torch.linalg.vector_norm(u) / torch.linalg.vector_norm(U)).item()
    # Gauss-Hermite weights w_j = W_j e^{-x_j^2} from the oracle's Hermite-function weights W
    # (numpy's hermgauss returns NaN weights at these sizes)
    ax = H.axis_1d(n)
    wt = torch.from_numpy(np.exp(ax.log_w - ax.x ** 2)).cuda()
    werr = torch.sqrt(torch.sum(wt[:, None, None] * wt[None, :, None] * wt[None, None, :] * u * u)).item()
    assert abs(err - rel_printed) < 0.006 * rel_printed, err
    assert abs(werr - w_printed) < 0.006 * w_printed, werr


def test_paper_table_magnus2_hermite_yoshida_dt02(T):
    """Table magnus2_hermite, Yoshida (M = 1), dt = 0.2, T = 1 (5 steps, 15 A-propagations)
    at the table's 499^3 Hermite grid, complex128 in FP64: error 1.34 (oracle, reduced to 1D:
    1.3379).  psi_0 = the ground state of -Delta + V1."""
    import torch
    n = 499
    x, _ = T.ts_grid_nodes(n, 1.0, -1)
    v1 = x ** 2 + 100 * np.sin(np.pi * x / 4) ** 2
    PA = T.ts_plan_create((n,) * 3, (1.0,) * 3, [np.zeros(n)] * 3, 0, order=-1)
    PH = T.ts_plan_create((n,) * 3, (1.0,) * 3, [v1] * 3, 0, order=-1)
    g = torch.from_numpy(T.ts_plan_eigvecs(PH, 0)[:, 0].copy()).cuda()
    g = g / torch.linalg.vector_norm(g)
    psi0 = (g[:, None, None] * g[None, :, None] * g[None, None, :]).reshape(-1).to(torch.complex128)
    v = torch.from_numpy(v1).cuda()
    VB = (v[:, None, None] + v[None, :, None] + v[None, None, :]).reshape(-1).contiguous()
    ref = torch.empty_like(psi0)
    T.ts_apply_exp(PH, 1.0, torch.view_as_real(psi0), torch.view_as_real(ref), T.TS_C128)
    psi = psi0.clone()
    na = T.ts_propagate(PA, T.TS_MAGNUS2, 1, 0.2, 5, VB, torch.view_as_real(psi), T.TS_C128)
    assert na == 15
    err = torch.linalg.vector_norm(psi - ref).item()
    assert abs(err - 1.34) < 0.006 * 1.34, err
