"""Helpers for the GPU parity tests: device tensors from numpy, plans on both sides."""
import numpy as np

import oracle as O
from paper_2605_20491_b300 import synth as S


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a = np.asarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.asarray(b, dtype=np.complex128 if cplx else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrel(a, b):
    """Max-norm error relative to the max-norm of the reference, ||a - b||_inf / ||b||_inf:
    beside the relative l2 error it catches an error confined to a few elements (one ragged
    tail tile), which the l2 norm of a large array would average away."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a = np.asarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.asarray(b, dtype=np.complex128 if cplx else np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# the max-norm bound of a parity test is MAXNORM_FACTOR times its relative l2 tolerance:
# a uniformly spread error of relative l2 size e has max-norm error up to a few e relative
# to the largest element, while one wrong tile gives a max-norm error near 1
MAXNORM_FACTOR = 20.0


def plans(n, L, f, mask=0):
    """(library plan, oracle plan) for the same grid and potential samples."""
    from paper_2605_20491_b300 import tschrod as T
    return T.ts_plan_create(n, L, f, mask), O.plan(n, L, f)


def harmonic_case(n, L=8.0, omega=None):
    d = len(n)
    Ls = (L,) * d
    om = omega if omega is not None else tuple(1.0 + 0.1 * k for k in range(d))
    return Ls, S.harmonic(n, Ls, om)
