"""Seeded synthetic inputs for the solver, shared by the oracle tests, the GPU tests
and the benchmark.

This module holds no arithmetic of the method itself: it only draws random numbers
and evaluates the problem's potentials and initial states at grid nodes.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  The generator seeded with ``seed`` returns as its
k-th output (k = 0, 1, ...) ``mix(seed + (k+1)*GAMMA)``, so any output can be computed
on its own; element ``idx`` of an array always uses the same outputs whatever the
array's length, which makes every input order-independent and reproducible.

* uniform on [lo, hi):  lo + (hi-lo) * (z >> 11) * 2^-53, output k = idx;
* standard normal:      Box-Muller on outputs 2*idx and 2*idx+1 (cosine branch);
* complex normal:       the cosine and sine branches of the same pair give re and im.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """k-th outputs (uint64) of the SplitMix64 generator seeded with ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (k + np.uint64(1)) * np.uint64(GAMMA)
        return _mix(z)


def splitmix64_scalar(seed: int, k: int) -> int:
    """Pure-integer SplitMix64 output, used to pin the vectorised version."""
    z = (seed + (k + 1) * GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def _unit(z: np.ndarray) -> np.ndarray:
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, _CHUNK):
        e = min(count, s + _CHUNK)
        k = np.arange(offset + s, offset + e, dtype=np.uint64)
        out[s:e] = lo + (hi - lo) * _unit(splitmix64(seed, k))
    return out


def _box_muller(seed: int, s: int, e: int):
    k = np.arange(s, e, dtype=np.uint64)
    u1 = 1.0 - _unit(splitmix64(seed, 2 * k))          # (0, 1]
    u2 = _unit(splitmix64(seed, 2 * k + np.uint64(1)))  # [0, 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad, 2.0 * math.pi * u2


def normal(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, _CHUNK):
        e = min(count, s + _CHUNK)
        rad, th = _box_muller(seed, s, e)
        out[s:e] = rad * np.cos(th)
    return out


def complex_normal(seed: int, count: int) -> np.ndarray:
    """Complex N(0,1)+iN(0,1), returned interleaved as float64 of length 2*count."""
    out = np.empty(2 * count, dtype=np.float64)
    for s in range(0, count, _CHUNK):
        e = min(count, s + _CHUNK)
        rad, th = _box_muller(seed, s, e)
        out[2 * s:2 * e:2] = rad * np.cos(th)
        out[2 * s + 1:2 * e:2] = rad * np.sin(th)
    return out


# ------------------------------------------- the same draws on a torch device -----
#
# For workloads too large to generate on the host in reasonable time (the serving
# benchmark's thousands of requests): SplitMix64 on int64 tensors, where multiplication
# wraps modulo 2^64 and logical right shifts are arithmetic shifts with the sign bits
# masked off.  The integer outputs equal splitmix64() bit for bit; the normals go through
# the device's log / cos / sin, which may differ from numpy's in the last bit.

def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(z, s: int):
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(seed: int, k):
    """splitmix64() on an int64 tensor of output indices k; int64 result with the same
    64 bits as the uint64 outputs."""
    z = _i64(seed & _MASK) + (k + 1) * _i64(GAMMA)
    z = (z ^ _srl(z, 30)) * _i64(_M1)
    z = (z ^ _srl(z, 27)) * _i64(_M2)
    return z ^ _srl(z, 31)


def _box_muller_torch(seed: int, count: int, device):
    import torch
    k = torch.arange(count, dtype=torch.int64, device=device)
    scale = 2.0 ** -53
    u1 = 1.0 - _srl(splitmix64_torch(seed, 2 * k), 11).to(torch.float64) * scale
    u2 = _srl(splitmix64_torch(seed, 2 * k + 1), 11).to(torch.float64) * scale
    return torch.sqrt(-2.0 * torch.log(u1)), 2.0 * math.pi * u2


def normal_torch(seed: int, count: int, device="cuda"):
    """normal() generated on `device` (float64 tensor)."""
    import torch
    rad, th = _box_muller_torch(seed, count, device)
    return rad * torch.cos(th)


def complex_normal_torch(seed: int, count: int, device="cuda"):
    """complex_normal() generated on `device`: interleaved float64 tensor of length 2 count."""
    import torch
    rad, th = _box_muller_torch(seed, count, device)
    return torch.stack((rad * torch.cos(th), rad * torch.sin(th)), dim=1).reshape(-1)


def v2_cos_bumps_torch(n, L, seed: int = 1, count: int = 8, device="cuda"):
    """v2_cos_bumps() evaluated on `device` (the bump parameters are drawn on the host)."""
    import torch
    assert len(n) == 3
    a, c = bumps_params(seed, count)
    x = [torch.from_numpy(_axis_coords(n, L, k)).to(device) for k in range(3)]
    v = 5.0 * torch.cos(x[0]) * torch.cos(x[1]) * torch.cos(x[2])
    for j in range(count):
        r2 = (x[0] - c[j][0]) ** 2 + (x[1] - c[j][1]) ** 2 + (x[2] - c[j][2]) ** 2
        v = v + a[j] * torch.exp(-r2)
    return v.reshape(-1).contiguous()


# ----------------------------------------------------------------- grids -----

def nodes(n: int, L: float) -> np.ndarray:
    """Coordinates of the n interior nodes of n+1 equal cells on [-L, L]."""
    h = 2.0 * L / (n + 1)
    return -L + h * np.arange(1, n + 1, dtype=np.float64)


def harmonic(n, L, omega):
    """Per-axis samples of V1 = sum_k (omega_k x_k)^2 at the nodes."""
    return [np.ascontiguousarray((om * nodes(nk, Lk)) ** 2) for nk, Lk, om in zip(n, L, omega)]


def _axis_coords(n, L, k):
    """Coordinate x_k of every grid point in vec() order (axis 0 fastest), as an array
    shaped for broadcasting."""
    shape = [1] * len(n)
    shape[k] = n[k]
    return nodes(n[k], L[k]).reshape(shape[::-1])


def bumps_params(seed: int, count: int = 8):
    """a_j ~ U[0,3), c_j ~ U[-4,4)^3 drawn in the order a_1, c_1, a_2, c_2, ..."""
    a, c = [], []
    k = 0
    for _ in range(count):
        a.append(float(uniform(seed, 1, 0.0, 3.0, offset=k)[0])); k += 1
        c.append([float(uniform(seed, 1, -4.0, 4.0, offset=k + j)[0]) for j in range(3)]); k += 3
    return np.array(a), np.array(c)


def v2_cos_bumps(n, L, seed: int = 1, count: int = 8) -> np.ndarray:
    """V2 = 5 cos x1 cos x2 cos x3 + sum_j a_j exp(-|x - c_j|^2) on a 3D grid, vec() order."""
    assert len(n) == 3
    a, c = bumps_params(seed, count)
    x = [_axis_coords(n, L, k) for k in range(3)]
    v = 5.0 * np.cos(x[0]) * np.cos(x[1]) * np.cos(x[2])
    for j in range(count):
        r2 = (x[0] - c[j][0]) ** 2 + (x[1] - c[j][1]) ** 2 + (x[2] - c[j][2]) ** 2
        v = v + a[j] * np.exp(-r2)
    return np.ascontiguousarray(v.reshape(-1))


def v2_soft_coulomb(n, L, strength: float = 1.0, delta: float = 1.0, dim: int = 3) -> np.ndarray:
    """V2 = sum_{i<j} c / sqrt(|r_i - r_j|^2 + delta^2) where particle i has the
    coordinates (x_{dim*i}, ..., x_{dim*i+dim-1}); vec() order, float64."""
    d = len(n)
    assert d % dim == 0
    P = d // dim
    x = [_axis_coords(n, L, k) for k in range(d)]
    v = np.zeros([n[k] for k in range(d)][::-1], dtype=np.float64)
    for i in range(P):
        for j in range(i + 1, P):
            r2 = 0.0
            for a in range(dim):
                r2 = r2 + (x[dim * i + a] - x[dim * j + a]) ** 2
            v = v + strength / np.sqrt(r2 + delta * delta)
    return np.ascontiguousarray(v.reshape(-1))


def sine_state(n, L) -> np.ndarray:
    """psi_0 = prod_k sin(pi (x_k + L_k) / (2 L_k)), normalised in l2, complex interleaved."""
    d = len(n)
    v = np.ones([n[k] for k in range(d)][::-1], dtype=np.float64)
    for k in range(d):
        v = v * np.sin(math.pi * (_axis_coords(n, L, k) + L[k]) / (2.0 * L[k]))
    v = v.reshape(-1)
    v = v / np.linalg.norm(v)
    out = np.zeros(2 * v.size)
    out[0::2] = v
    return out


# ------------------------------------------------------------ workloads -----

#: The five workloads the library is exercised on (sizes, domains, potentials, seeds).
WORKLOADS = {
    "3d_n32_fp64": dict(d=3, n=(32, 32, 32), L=(8.0,) * 3, omega=(1.0, 1.0, 1.0), sigma=1.0,
                        rhs="uniform", seed=0, lu_n=8),
    "3d_n512_apply": dict(d=3, n=(512, 512, 512), L=(8.0,) * 3, omega=(1.0, 1.3, 0.7), sigma=0.5,
                          rhs="normal", seed=2, psi_seed=3, tau=0.01),
    "3d_n256_pcg": dict(d=3, n=(256, 256, 256), L=(8.0,) * 3, omega=(1.0, 1.0, 1.0), v2_seed=1,
                        pcg_tol=1e-10, lambda_tol=1e-12),
    "6d_n24_strang": dict(d=6, n=(24,) * 6, L=(5.0,) * 6, omega=(1.0,) * 6, dt=0.01, steps=100),
    "9d_n8_strang": dict(d=9, n=(8,) * 9, L=(3.0,) * 9, omega=(1.0,) * 9, dt=0.01, steps=100),
}


def serving_requests(count: int, seed: int = 4, sizes=(32, 48, 64, 96, 128), omega_set=None,
                     mix=(0.3, 0.5, 0.2)):
    """Request descriptors of the serving workload: per request, n_k i.i.d. from `sizes` per
    axis (3D), L = 8, sigma ~ U[0.5, 5), omega_k ~ U[0.5, 2) (or drawn from omega_set),
    kind PCG / inverse / exp with probabilities `mix`, tau = 0.01, right-hand side seed
    1000 + id.  Draws come from SplitMix64(seed) in a fixed order per request."""
    out = []
    k = 0
    def u(lo=0.0, hi=1.0):
        nonlocal k
        v = float(uniform(seed, 1, lo, hi, offset=k)[0])
        k += 1
        return v
    for rid in range(count):
        n = tuple(sizes[min(int(u() * len(sizes)), len(sizes) - 1)] for _ in range(3))
        sigma = u(0.5, 5.0)
        if omega_set:
            omega = tuple(omega_set[min(int(u() * len(omega_set)), len(omega_set) - 1)] for _ in range(3))
        else:
            omega = tuple(u(0.5, 2.0) for _ in range(3))
        r = u()
        kind = "pcg" if r < mix[0] else ("inverse" if r < mix[0] + mix[1] else "exp")
        out.append(dict(id=rid, kind=kind, n=n, L=(8.0, 8.0, 8.0), omega=omega, sigma=sigma, tau=0.01,
                        rhs_seed=1000 + rid))
    return out
