// Pointwise kernels of the solver: the eigenvalue scale (step 3 of Sec. 2.1), the
// propagator phase e^{-i tau Lambda} (eq. exact_prop), the potential phase e^{-i V2 theta}
// of the Strang step (Sec. 5.1), the 2d+1 point operator of eq. general_system, the
// PCG vector updates (Sec. 3.2) and deterministic FP64 reductions.
//
// All kernels are HBM-bound streams; they use grid-stride loops over a fixed grid of
// (148 SMs x 4) CTAs so that reductions see a fixed partition of the index space and
// return bit-identical sums on every call (two-level reduction: per-CTA partials in a
// fixed order, then one CTA sums the partials in a fixed order).
#include <algorithm>
#include <vector>

#include "async_copy.cuh"
#include "common.cuh"
#include "fixed.cuh"
#include "pointwise.cuh"
#include "sem_axis.cuh"
#include "split.cuh"

namespace ts {

AxisParams axis_params(const ts_plan* p, bool eig_tables) {
  AxisParams a{};
  a.d = p->d;
  long long st = 1;
  for (int k = 0; k < p->d; ++k) {
    a.n[k] = p->n[k];
    a.stride[k] = st;
    st *= p->n[k];
    double h = 2.0 * p->L[k] / (p->n[k] + 1);
    a.ih2[k] = 1.0 / (h * h);
    a.tab[k] = eig_tables ? p->lam[k] : p->f[k];
  }
  return a;
}

namespace {

__device__ __forceinline__ double lambda_sum(const AxisParams& a, long long idx) {
  double s = 0.0;
  for (int k = 0; k < a.d; ++k) {
    long long q = idx / a.n[k];
    int i = (int)(idx - q * a.n[k]);
    s += a.tab[k][i];
    idx = q;
  }
  return s;
}

__global__ void k_scale_inverse(AxisParams a, double sigma, double* X, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    X[i] = X[i] / (lambda_sum(a, i) + sigma);
}

__global__ void k_scale_exp(AxisParams a, double tau, double* X, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s, c;
    sincos(tau * lambda_sum(a, i), &s, &c);
    double re = X[2 * i], im = X[2 * i + 1];
    X[2 * i] = re * c + im * s;
    X[2 * i + 1] = im * c - re * s;
  }
}

__global__ void k_phase_c128(const double* V2, double th, double* psi, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s, c;
    sincos(th * V2[i], &s, &c);
    double re = psi[2 * i], im = psi[2 * i + 1];
    psi[2 * i] = re * c + im * s;
    psi[2 * i + 1] = im * c - re * s;
  }
}

__global__ void k_phase_c64(const double* V2, double th, float* psi, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s, c;
    sincos(th * V2[i], &s, &c);
    float2 v = reinterpret_cast<float2*>(psi)[i];
    float re = v.x, im = v.y;
    reinterpret_cast<float2*>(psi)[i] = make_float2((float)(re * c + im * s), (float)(im * c - re * s));
  }
}

__global__ void k_c64_to_c128(const float* in, double* out, long long n2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

__global__ void k_c128_to_c64(const double* in, float* out, long long n2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// ---------------------------------------------------------------- reductions ---

// Block-wide sum in a fixed order: warp shuffles then one warp over the warp sums.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? ws[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// The 2d+1 point operator of eq. general_system, A x = sum_k h_k^-2 (2x - x_{-e_k} - x_{+e_k})
// + (sigma + V1 + V2) x with zero Dirichlet ghosts, in three forms:
//   MODE 0: y = A x;                      partial sums of x.y
//   MODE 1: y = b - A x;                  partial sums of y.y and b.b
//   MODE 2: planes = split(b - A x);      partial sums of (b - A x)^2 and b.b
// Work is mapped by grid rows (all axes but the first): a group of G lanes (G = n_1
// rounded up to a power of two, at most 32) walks one row with unit stride, so the
// multi-index of the row is decomposed once per row and every load is coalesced.
template <int MODE, int NP>
__global__ void k_stencil(AxisParams a, const double* __restrict__ V2, double sigma, const double* __restrict__ x,
                          const double* __restrict__ b, double* __restrict__ y, __nv_bfloat16* __restrict__ planes,
                          long long N, double* partial) {
  // FP64 instructions are the scarce resource on this GPU (about two per clock per SM),
  // so the operator is evaluated as  A x = diag x - sum_k h_k^-2 (x_{-e_k} + x_{+e_k})
  // with diag = sigma + V1 + V2 + 2 sum_k h_k^-2 (the row part summed once per row):
  // about 2 FP64 instructions per axis and element.
  const int n0 = a.n[0];
  int G = 1;
  while (G < n0 && G < 32) G <<= 1;
  const int rows_per_warp = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const long long R = N / n0;
  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double c0 = a.ih2[0];
  double acc0 = 0.0, acc1 = 0.0;
  for (long long rb = wid * rows_per_warp; rb < R; rb += warps_total * rows_per_warp) {
    const long long row = rb + sub;
    if (row >= R) continue;
    long long q = row;
    double drow = sigma + 2.0 * c0;
    unsigned lo_mask = 0, hi_mask = 0;
    for (int k = 1; k < a.d; ++k) {
      long long qq = q / a.n[k];
      int i = (int)(q - qq * a.n[k]);
      q = qq;
      drow += a.tab[k][i] + 2.0 * a.ih2[k];
      if (i == 0) lo_mask |= 1u << k;
      if (i == a.n[k] - 1) hi_mask |= 1u << k;
    }
    const long long base = row * n0;
    for (int i0 = gl; i0 < n0; i0 += G) {
      const long long idx = base + i0;
      const double xc = x[idx];
      double diag = drow + a.tab[0][i0];
      if (V2) diag += V2[idx];
      const double l0 = i0 > 0 ? x[idx - 1] : 0.0;
      const double r0 = i0 + 1 < n0 ? x[idx + 1] : 0.0;
      // MODE 0: acc = A x;  MODE 1, 2: acc = b - A x
      double acc = MODE == 0 ? diag * xc : fma(-diag, xc, b[idx]);
      const double sgn = MODE == 0 ? -1.0 : 1.0;
      acc = fma(sgn * c0, l0 + r0, acc);
      for (int k = 1; k < a.d; ++k) {
        const double left = ((lo_mask >> k) & 1u) ? 0.0 : x[idx - a.stride[k]];
        const double right = ((hi_mask >> k) & 1u) ? 0.0 : x[idx + a.stride[k]];
        acc = fma(sgn * a.ih2[k], left + right, acc);
      }
      if (MODE == 0) {
        y[idx] = acc;
        acc0 = fma(xc, acc, acc0);
      } else if (MODE == 1) {
        y[idx] = acc;
        const double bi = b[idx];
        acc0 = fma(acc, acc, acc0);
        acc1 = fma(bi, bi, acc1);
      } else {  // planes: rows of axis 1 padded to a multiple of 8
        split_store<NP>((float)acc, planes, R * ((n0 + 7) & ~7), row * ((n0 + 7) & ~7) + i0);
      }
    }
  }
  if (MODE == 2) return;  // the refinement needs no norms
  double s0 = block_sum(acc0);
  double s1 = block_sum(acc1);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// Residual r = b - (-Delta_h + V1 + sigma) u split into bf16 planes, for grids with the
// same h on every axis.  The Laplacian part sum_k (2u - u_{-e_k} - u_{+e_k}) -- where all the
// cancellation happens -- is evaluated exactly in 64-bit fixed point (one global scale from
// the largest exponent of u, headroom H bits so that 4d |U| < 2^63); the rest is FP64:
//   r = (b - (sigma + V1) u) - h^-2 2^(emax - 1022 - H) * L_int.
// About 5 FP64-pipe instructions per point instead of 9; the integer work runs on the
// otherwise idle integer pipe.
template <int NP>
__global__ void k_residual_fixed(AxisParams a, double sigma, const double* __restrict__ x,
                                 const double* __restrict__ b, __nv_bfloat16* __restrict__ planes, long long N,
                                 const int* __restrict__ emax_ptr, int H) {
  const int emax = *emax_ptr;
  const double cs = ldexp(a.ih2[0], emax - 1022 - H);
  const int P = H - 53;
  const int n0 = a.n[0];
  int G = 1;
  while (G < n0 && G < 32) G <<= 1;
  const int rows_per_warp = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const long long R = N / n0;
  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long twod = 2LL * a.d;
  for (long long rb = wid * rows_per_warp; rb < R; rb += warps_total * rows_per_warp) {
    const long long row = rb + sub;
    if (row >= R) continue;
    long long q = row;
    double drow = sigma;
    unsigned lo_mask = 0, hi_mask = 0;
    for (int k = 1; k < a.d; ++k) {
      long long qq = q / a.n[k];
      int i = (int)(q - qq * a.n[k]);
      q = qq;
      drow += a.tab[k][i];
      if (i == 0) lo_mask |= 1u << k;
      if (i == a.n[k] - 1) hi_mask |= 1u << k;
    }
    const long long base = row * n0;
    for (int i0 = gl; i0 < n0; i0 += G) {
      const long long idx = base + i0;
      const double xc = x[idx];
      long long L = twod * to_fixed(xc, emax, P);
      if (i0 > 0) L -= to_fixed(x[idx - 1], emax, P);
      if (i0 + 1 < n0) L -= to_fixed(x[idx + 1], emax, P);
      for (int k = 1; k < a.d; ++k) {
        if (!((lo_mask >> k) & 1u)) L -= to_fixed(x[idx - a.stride[k]], emax, P);
        if (!((hi_mask >> k) & 1u)) L -= to_fixed(x[idx + a.stride[k]], emax, P);
      }
      const double diag = drow + a.tab[0][i0];
      const double r = fma(-cs, __ll2double_rn(L), fma(-diag, xc, b[idx]));
      split_store<NP>((float)r, planes, R * ((n0 + 7) & ~7), row * ((n0 + 7) & ~7) + i0);
    }
  }
}

// Q tables of the folded diagonal: Q[0] = sigma / h^-2, then f_0 / h^-2, f_1 / h^-2,
// f_2 / h^-2, each as a fixed-point integer with F fractional bits (rounded to nearest).
__global__ void k_qtables(const double* f0, int n0, const double* f1, int n1, const double* f2, int n2, double sigma,
                          double ih2, int F, long long* Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = 1 + n0 + n1 + n2;
  if (i >= total) return;
  double v;
  if (i == 0) v = sigma;
  else if (i <= n0) v = f0[i - 1];
  else if (i <= n0 + n1) v = f1[i - 1 - n0];
  else v = f2[i - 1 - n0 - n1];
  Q[i] = llrint(ldexp(v / ih2, F));
}

// The same residual for d = 3, converting every value to fixed point once: a block owns a
// 32 x 16 tile of axes (0, 1) and marches along axis 2 over MZ planes.  The axis-2 neighbours
// come from a three-plane register queue; the axis-0/1 neighbours from a shared-memory copy
// of the current plane with a one-cell halo (converted by warps 0-2: top row, bottom row,
// left and right columns).  Loads run RD - 1 steps ahead through a per-thread ring in
// shared memory filled by cp.async (each thread lands exactly the values it reads later:
// its two cells of x and b and its halo cell), so that enough bytes are in flight to cover
// HBM latency without holding them in registers.  The conversion of the residual to float
// runs on the integer pipe.
// QF = false: H = 58 (4d |U| < 2^62); three FP64 instructions per point remain (diagonal
//   sum, two FMAs).
// QF = true: the diagonal (sigma + V1) u joins the fixed-point sum as (Q_a + Q_z) U >> F,
//   with Q = (sigma + f_0 + f_1) / h^-2 per thread and f_2 / h^-2 per plane from the Q
//   tables (F fractional bits) and a 128-bit integer product; H = 53 + P leaves room for
//   4d |U| + |Q U| / 2^F.  One FP64 instruction per point remains: r = b - c_s L.
constexpr int MX = 32, MY = 16, MZ = 32;
constexpr int RD = 4;           // ring depth (groups in flight: RD - 1)
constexpr int RING_VALUES = 5;  // per thread and group: x(z+1) of both cells, halo x(z+1), b(z) of both cells
constexpr int RING_BYTES = RD * RING_VALUES * 256 * 8;
// APPLY (with QF): the operator itself for PCG, y = A x = c_s L + V2 x, where b carries
//   V2 (NULL: none) and y is written in FP64 to `yout`; each block adds x.y into
//   partial[2 blockIdx], partial[2 blockIdx + 1] = 0 (summed in a fixed order afterwards).
template <int NP, int P, bool QF, bool APPLY = false>
__global__ void __launch_bounds__(256) k_residual_march3(AxisParams a, double sigma, const long long* __restrict__ Q,
                                                         int F, const double* __restrict__ x,
                                                         const double* __restrict__ b,
                                                         __nv_bfloat16* __restrict__ planes, long long N,
                                                         const int* __restrict__ emax_ptr, double* yout = nullptr,
                                                         double* partial = nullptr) {
  static_assert(!APPLY || QF, "the operator form folds the separable diagonal");
  constexpr int H = 53 + P;
  double dot = 0.0;
  __shared__ long long sU[2][MY + 2][MX + 2];
  const int emax = *emax_ptr;
  const double cs = ldexp(a.ih2[0], emax - 1022 - H);
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const long long s2 = (long long)n0 * n1;
  const int tiles0 = (n0 + MX - 1) / MX, tiles1 = (n1 + MY - 1) / MY;
  int bid = blockIdx.x;
  const int t0 = bid % tiles0;
  bid /= tiles0;
  const int t1 = bid % tiles1;
  const int z0 = (bid / tiles1) * MZ, z1 = min(z0 + MZ, n2);
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int i0 = t0 * MX + lx;
  const int ia = t1 * MY + ly, ib = ia + 8;
  const bool va = i0 < n0 && ia < n1, vb = i0 < n0 && ib < n1;
  const long long oa = (long long)ia * n0 + i0, ob = (long long)ib * n0 + i0;
  // halo cell of this thread (warps 0-2): smem (hy, hx), grid (hi0, hi1)
  int hy = 0, hx = 0, hi0 = -1, hi1 = -1;
  if (ly == 0) { hy = 0; hx = lx + 1; hi0 = i0; hi1 = t1 * MY - 1; }
  else if (ly == 1) { hy = MY + 1; hx = lx + 1; hi0 = i0; hi1 = t1 * MY + MY; }
  else if (ly == 2) {
    hy = (lx & 15) + 1;
    hx = lx < 16 ? 0 : MX + 1;
    hi0 = lx < 16 ? t0 * MX - 1 : t0 * MX + MX;
    hi1 = t1 * MY + (lx & 15);
  }
  const bool hv = ly < 3 && hi0 >= 0 && hi0 < n0 && hi1 >= 0 && hi1 < n1;
  const long long oh = hv ? (long long)hi1 * n0 + hi0 : 0;
  const double ca = !QF && va ? sigma + a.tab[0][i0] + a.tab[1][ia] : 0.0;
  const double cb = !QF && vb ? sigma + a.tab[0][i0] + a.tab[1][ib] : 0.0;
  const long long qa = QF && va ? Q[0] + Q[1 + i0] + Q[1 + n0 + ia] : 0;
  const long long qb = QF && vb ? Q[0] + Q[1 + i0] + Q[1 + n0 + ib] : 0;
  const double* f2 = a.tab[2];
  const long long* q2 = QF ? Q + 1 + n0 + n1 : nullptr;

  // ring[g][v][thread]: group g % RD, value v (0, 1: x of cells a, b at z + 1; 2: halo x at
  // z + 1; 3, 4: b of cells a, b at z), consecutive threads in consecutive words
  static_assert((RD & (RD - 1)) == 0, "ring depth is a power of two");
  extern __shared__ double ring[];
  double* const my_ring = ring + threadIdx.x;
  // group of step z: x(z + 1) of both cells and of the halo cell, b(z) of both cells;
  // out-of-range values are zero-filled (Dirichlet zeros outside the grid).  Source
  // pointers advance by one plane per issued group; invalid cells read nothing.
  const double* sxa = x + (va ? oa + (long long)(z0 + 1) * s2 : 0);
  const double* sxb = x + (vb ? ob + (long long)(z0 + 1) * s2 : 0);
  const double* sxh = x + (hv ? oh + (long long)(z0 + 1) * s2 : 0);
  const double* sba = b ? b + (va ? oa + (long long)z0 * s2 : 0) : nullptr;
  const double* sbb = b ? b + (vb ? ob + (long long)z0 * s2 : 0) : nullptr;
  const long long sa_step = va ? s2 : 0, sb_step = vb ? s2 : 0, sh_step = hv ? s2 : 0;
  auto issue = [&](int z) {
    if (z < z1) {
      double* dst = my_ring + ((z - z0) & (RD - 1)) * (RING_VALUES * 256);
      const bool xn = z + 1 < n2, hn = hv && z + 1 < z1;
      cp_async8_zfill(dst, va && xn ? sxa : x, va && xn);  // past the last plane: no address
      cp_async8_zfill(dst + 256, vb && xn ? sxb : x, vb && xn);
      if (ly < 3) cp_async8_zfill(dst + 512, hn ? sxh : x, hn);
      cp_async8_zfill(dst + 768, b && va ? sba : x, b && va);
      cp_async8_zfill(dst + 1024, b && vb ? sbb : x, b && vb);
      sxa += sa_step;
      sxb += sb_step;
      sxh += sh_step;
      if (b) {
        sba += sa_step;
        sbb += sb_step;
      }
    }
    cp_async_commit();  // an empty group past the end keeps the group count uniform
  };
  for (int k = 0; k < RD - 1; ++k) issue(z0 + k);
  // output pointers of the two cells' plane-0 elements, advanced one z-slab per step; the
  // planes' rows (axis 1) are padded to ld0 elements, a multiple of 8
  const int ld0 = (n0 + 7) & ~7;
  const long long ps2 = (long long)ld0 * n1;
  const long long Np = ps2 * n2;
  __nv_bfloat16* pa = planes + (va ? (long long)ia * ld0 + i0 + (long long)z0 * ps2 : 0);
  __nv_bfloat16* pb = planes + (vb ? (long long)ib * ld0 + i0 + (long long)z0 * ps2 : 0);
  auto ld = [&](bool v, const double* base, long long off, int z) -> double {
    return v ? base[off + z * s2] : 0.0;
  };
  long long Upa = to_fixed(ld(va && z0 > 0, x, oa, z0 - 1), emax, P);
  long long Upb = to_fixed(ld(vb && z0 > 0, x, ob, z0 - 1), emax, P);
  double xca = ld(va, x, oa, z0), xcb = ld(vb, x, ob, z0);
  long long Uca = to_fixed(xca, emax, P), Ucb = to_fixed(xcb, emax, P);
  sU[0][ly + 1][lx + 1] = Uca;
  sU[0][ly + 9][lx + 1] = Ucb;
  if (ly < 3) sU[0][hy][hx] = to_fixed(ld(hv, x, oh, z0), emax, P);
  int buf = 0;
  for (int z = z0; z < z1; ++z) {
    cp_async_wait<RD - 2>();  // this step's group has landed (this thread's own copies)
    const double* src = my_ring + ((z - z0) & (RD - 1)) * (RING_VALUES * 256);
    const double xna = src[0], xnb = src[256];
    const double xnh = ly < 3 ? src[512] : 0.0;
    const double b_a = src[768], b_b = src[1024];
    issue(z + RD - 1);  // refills the slot read in the previous step (by this same thread)
    const long long Una = to_fixed(xna, emax, P), Unb = to_fixed(xnb, emax, P);
    const long long Unh = to_fixed(xnh, emax, P);
    const double xa = xca, xb = xcb;
    xca = xna;
    xcb = xnb;
    __syncthreads();
    const long long(*T)[MX + 2] = sU[buf];
    const long long La = 6 * Uca - Upa - Una - T[ly + 1][lx] - T[ly + 1][lx + 2] - T[ly][lx + 1] - T[ly + 2][lx + 1];
    const long long Lb = 6 * Ucb - Upb - Unb - T[ly + 9][lx] - T[ly + 9][lx + 2] - T[ly + 8][lx + 1] -
                         T[ly + 10][lx + 1];
    if (APPLY) {
      const long long qz = q2[z];
      const long long zoff = (long long)z * s2;
      if (va) {
        const double y = fma(b_a, xa, cs * __ll2double_rn(La + mul_shift(qa + qz, Uca, F)));
        yout[oa + zoff] = y;
        dot = fma(xa, y, dot);
      }
      if (vb) {
        const double y = fma(b_b, xb, cs * __ll2double_rn(Lb + mul_shift(qb + qz, Ucb, F)));
        yout[ob + zoff] = y;
        dot = fma(xb, y, dot);
      }
    } else if (QF) {
      const long long qz = q2[z];
      if (va) {
        const double r = fma(-cs, __ll2double_rn(La + mul_shift(qa + qz, Uca, F)), b_a);
        split_store<NP>(f64_to_f32(r), pa, Np, 0);
      }
      if (vb) {
        const double r = fma(-cs, __ll2double_rn(Lb + mul_shift(qb + qz, Ucb, F)), b_b);
        split_store<NP>(f64_to_f32(r), pb, Np, 0);
      }
    } else {
      const double fz = f2[z];
      if (va) {
        const double r = fma(-cs, i64_to_f64(La), fma(-(ca + fz), xa, b_a));
        split_store<NP>(f64_to_f32(r), pa, Np, 0);
      }
      if (vb) {
        const double r = fma(-cs, i64_to_f64(Lb), fma(-(cb + fz), xb, b_b));
        split_store<NP>(f64_to_f32(r), pb, Np, 0);
      }
    }
    pa += va ? ps2 : 0;
    pb += vb ? ps2 : 0;
    sU[buf ^ 1][ly + 1][lx + 1] = Una;
    sU[buf ^ 1][ly + 9][lx + 1] = Unb;
    if (ly < 3) sU[buf ^ 1][hy][hx] = Unh;
    Upa = Uca;
    Upb = Ucb;
    Uca = Una;
    Ucb = Unb;
    buf ^= 1;
  }
  if (APPLY) {
    dot = block_sum(dot);
    if (threadIdx.x == 0) {
      partial[2 * blockIdx.x] = dot;
      partial[2 * blockIdx.x + 1] = 0.0;
    }
  }
}

// partial sums of (a.b) and (c.d) (c, d may be NULL).
__global__ void k_dot2(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                       const double* __restrict__ d, long long N, double* partial) {
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    s0 += b ? a[i] * b[i] : a[i];
    if (c) s1 += c[i] * d[i];
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// r = b - y (y = A x already in r) with partial sums of r.r and b.b.
__global__ void k_sub_dot(const double* __restrict__ b, double* __restrict__ r, long long N, double* partial) {
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double v = bi - r[i];
    r[i] = v;
    s0 += v * v;
    s1 += bi * bi;
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// Sum the partials in a fixed order; out[0], out[1] = the two sums.
__global__ void k_sum_partials(const double* partial, int nblk, double* out) {
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    s0 += partial[2 * i];
    s1 += partial[2 * i + 1];
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
  }
}

// PCG step: alpha = rz / pq; x += alpha p; r -= alpha q; partial r.r; alpha -> *alpha_out.
__global__ void k_pcg_xr(const double* rz, const double* pq, double* alpha_out, double* __restrict__ x,
                         double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q,
                         long long N, double* partial) {
  // a zero p.q only arises after exact convergence (p = 0): then no step (also for the
  // extra iteration that the lagged stopping test may run)
  double alpha = pq[0] != 0.0 ? rz[0] / pq[0] : 0.0;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    acc += ri * ri;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = acc;
    partial[2 * blockIdx.x + 1] = 0.0;
    if (blockIdx.x == 0) *alpha_out = alpha;
  }
}

// p = z + beta p with the flexible beta = -alpha (z_{k+1}.q_k) / (z_k.r_k); first: p = z.
// emax_out (may be NULL): raised to the largest biased exponent of the new p.
__global__ void k_pcg_p(const double* alpha, const double* zq, const double* rz_old, int first,
                        double* __restrict__ p, const double* __restrict__ z, long long N, int* emax_out) {
  double beta = first || rz_old[0] == 0.0 ? 0.0 : -alpha[0] * zq[0] / rz_old[0];
  int emx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = first ? z[i] : fma(beta, p[i], z[i]);
    p[i] = v;
    emx = max(emx, (__double2hiint(v) >> 20) & 0x7FF);
  }
  if (emax_out) {
    for (int o = 16; o > 0; o >>= 1) emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(emax_out, emx);
  }
}

__global__ void k_copy_scalar(const double* src, double* dst) { *dst = *src; }

// u = prod_k g_k[i_k] where g_k = row 0 of S_k^T (the ground eigenvector of axis k).
__global__ void k_tensor_ground(AxisParams a, double* u, long long N) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    double v = 1.0;
    for (int k = 0; k < a.d; ++k) {
      long long q = r / a.n[k];
      int i = (int)(r - q * a.n[k]);
      r = q;
      v *= a.tab[k][i];
    }
    u[idx] = v;
  }
}

// y = a x + b y; with b == 0, y is not read (BLAS convention): it may hold anything, e.g. a
// recycled scratch buffer whose stale bits form NaNs.
__global__ void k_axpby(double a, const double* x, double b, double* y, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(b, y[i], a * x[i]);
}

__global__ void k_scale_by_scalar(const double* num, const double* den, double* y, const double* x, long long N) {
  // y = x * (num[0] / den[0]) -- den may be NULL (then y = x / sqrt(num[0]))
  double f = den ? num[0] / den[0] : 1.0 / sqrt(num[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

// Per-axis band tables of a Q^k plan (k >= 2), by value.
struct BandParams {
  int d;
  int order;                  // k of Q^k (>= 2), or -1 (Hermite: dense rows)
  int w[MAXD];                // half bandwidth per axis (k of Q^k; n - 1 for Hermite)
  int n[MAXD];
  long long stride[MAXD];
  const double* band[MAXD];   // n[k] rows of 2w + 1: band[i][o] = K[i][i + o - w]
  const double* f[MAXD];      // V1 samples
};

// The Q^k operator of eq. general_system, A x = sum_k K_k x (along axis k) + (sigma + V1 + V2) x,
// with K_k banded (half bandwidth w = k; M^{-1} Stiff, or M^{-1/2} Stiff M^{-1/2} in the
// symmetric frame), in the three forms of k_stencil (MODE 0: y = A x and x.y; MODE 1:
// y = b - A x, y.y and b.b; MODE 2: split(b - A x) into bf16 planes).  Same mapping as
// k_stencil: G lanes walk one grid row (axis 1) with unit stride, the multi-index of the row
// is decomposed once per row and the band rows of the other axes are the same for the whole
// row.  Structural zeros of Q^k rows are skipped on every axis: about d (k + 2) FP64
// multiply-adds per point instead of d (2k + 1).
template <int MODE, int NP>
__global__ void k_banded(BandParams a, const double* __restrict__ V2, double sigma, const double* __restrict__ x,
                         const double* __restrict__ b, double* __restrict__ y, __nv_bfloat16* __restrict__ planes,
                         long long N, double* partial) {
  const int n0 = a.n[0], w = a.w[0], bw = 2 * a.w[0] + 1;
  int G = 1;
  while (G < n0 && G < 32) G <<= 1;
  const int rows_per_warp = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
  const long long R = N / n0;
  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double acc0 = 0.0, acc1 = 0.0;
  for (long long rb = wid * rows_per_warp; rb < R; rb += warps_total * rows_per_warp) {
    const long long row = rb + sub;
    if (row >= R) continue;
    long long q = row;
    double drow = sigma;
    int ik[MAXD];
    for (int k = 1; k < a.d; ++k) {
      const long long qq = q / a.n[k];
      ik[k] = (int)(q - qq * a.n[k]);
      q = qq;
      drow += a.f[k][ik[k]];
    }
    const long long base = row * n0;
    // one node: axis-1 band entries olo..ohi (clipped to the row), then the other axes
    auto node = [&](int i0, int olo, int ohi) {
      const long long idx = base + i0;
      double diag = drow + a.f[0][i0];
      if (V2) diag += V2[idx];
      double ax = diag * x[idx];
      {
        const double* B = a.band[0] + (long long)i0 * bw;
        const int lo = max(olo, i0 - w < 0 ? w - i0 : 0), hi = min(ohi, i0 + w >= n0 ? w + n0 - 1 - i0 : 2 * w);
        for (int o = lo; o <= hi; ++o) ax = fma(B[o], x[idx + o - w], ax);
      }
      for (int k = 1; k < a.d; ++k) {
        // the row index is the same for all lanes here, so the element structure of Q^k is
        // used to skip the band's structural zeros: node g = i + 1 at position p = g mod k of
        // its element couples to that element's k + 1 nodes only (o in [k - p, 2k - p]) unless
        // it is a shared element end (p = 0: both elements, the full band)
        const int wk = a.w[k];
        const double* B = a.band[k] + (long long)ik[k] * (2 * wk + 1);
        int lo = ik[k] - wk < 0 ? wk - ik[k] : 0, hi = ik[k] + wk >= a.n[k] ? wk + a.n[k] - 1 - ik[k] : 2 * wk;
        if (a.order >= 2) {
          const int pos = (ik[k] + 1) % a.order;
          if (pos != 0) {
            lo = max(lo, a.order - pos);
            hi = min(hi, 2 * a.order - pos);
          }
        }
        const long long st = a.stride[k];
        for (int o = lo; o <= hi; ++o) ax = fma(B[o], x[idx + (o - wk) * st], ax);
      }
      if (MODE == 0) {
        y[idx] = ax;
        acc0 = fma(x[idx], ax, acc0);
      } else {
        const double bi = b[idx];
        const double r = bi - ax;
        if (MODE == 1) {
          y[idx] = r;
          acc0 = fma(r, r, acc0);
          acc1 = fma(bi, bi, acc1);
        } else {  // planes: rows of axis 1 padded to a multiple of 8
          split_store<NP>((float)r, planes, R * ((n0 + 7) & ~7), row * ((n0 + 7) & ~7) + i0);
        }
      }
    };
    if (a.order >= 2) {
      // Q^k rows in two uniform loops, so that lanes do not wait on each other: the
      // element-interior nodes (k - 1 per element, node g = i0 + 1 at position p = g mod k)
      // couple to their element's k + 1 nodes, band entries k - p .. 2k - p; the shared
      // element ends (p = 0, every k-th node) to both elements, the full band.
      const int kq = a.order;
      const int nb = (n0 + 1) / kq - 1;  // shared element ends in the row
      for (int j = gl; j < n0 - nb; j += G) {
        const int i0 = j + j / (kq - 1);
        const int pos = (i0 + 1) % kq;
        node(i0, kq - pos, 2 * kq - pos);
      }
      for (int m = gl; m < nb; m += G) node((m + 1) * kq - 1, 0, 2 * w);
    } else {
      for (int i0 = gl; i0 < n0; i0 += G) node(i0, 0, 2 * w);
    }
  }
  if (MODE == 2) return;
  double s0 = block_sum(acc0);
  double s1 = block_sum(acc1);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// y = x * prod_k tab_k[i_k] (a separable diagonal, e.g. M^{1/2} or M^{-1/2}); x and y may alias.
__global__ void k_scale_separable(AxisParams a, const double* x, double* y, long long N) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    long long q = idx;
    double s = 1.0;
    for (int k = 0; k < a.d; ++k) {
      const long long qq = q / a.n[k];
      s *= a.tab[k][(int)(q - qq * a.n[k])];
      q = qq;
    }
    y[idx] = x[idx] * s;
  }
}

// Per-axis quadrature weights of the L2 inner product: w_k(i) = mh_k[i]^2 (Q^k: the GLL
// lumped mass) or h_k (Q^1, mh_k == NULL); the d-dimensional weight is their product.
struct WeightParams {
  int d;
  int n[MAXD];
  const double* mh[MAXD];
  double h[MAXD];
};

__device__ __forceinline__ double axis_weight(const WeightParams& w, int k, int i) {
  if (w.mh[k]) {
    const double m = w.mh[k][i];
    return m * m;
  }
  return w.h[k];
}

// Weighted reductions over grid rows (axis 1): one warp per row, the weight of the row's
// other axes computed once.  MODE 0: sums of W a b and W c d (c may be NULL); MODE 1: sums
// of W a b and W a^4 (the GPE energy terms, a = u, b = H_u u); MODE 2: sum of W (b - s a)^2
// (the Euler-Lagrange residual, s = lambda).
template <int MODE>
__global__ void k_wdot(WeightParams w, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, const double* __restrict__ dv, long long N, double* partial,
                       double sc = 0.0) {
  const int n0 = w.n[0];
  const long long R = N / n0;
  const int lane = threadIdx.x & 31;
  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  double s0 = 0.0, s1 = 0.0;
  for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < R; row += warps_total) {
    long long q = row;
    double wr = 1.0;
    for (int k = 1; k < w.d; ++k) {
      const long long qq = q / w.n[k];
      wr *= axis_weight(w, k, (int)(q - qq * w.n[k]));
      q = qq;
    }
    const long long base = row * n0;
    for (int i0 = lane; i0 < n0; i0 += 32) {
      const long long idx = base + i0;
      const double wt = wr * axis_weight(w, 0, i0);
      const double av = a[idx];
      if (MODE == 2) {
        const double e = fma(-sc, av, b[idx]);
        s0 = fma(wt * e, e, s0);
        continue;
      }
      s0 = fma(wt * av, b[idx], s0);
      if (MODE == 1) {
        const double a2 = av * av;
        s1 = fma(wt * a2, a2, s1);
      } else if (c) {
        s1 = fma(wt * c[idx], dv[idx], s1);
      }
    }
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// veff = V2 + beta u^2 (V2 may be NULL).
__global__ void k_gpe_veff(const double* __restrict__ V2, double beta, const double* __restrict__ u,
                           double* __restrict__ veff, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double ui = u[i];
    veff[i] = fma(beta * ui, ui, V2 ? V2[i] : 0.0);
  }
}

// u = u + a x + b y.
__global__ void k_axpy2(double* __restrict__ u, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    u[i] = fma(b, y[i], fma(a, x[i], u[i]));
}

// Tensor-product linear interpolation from a coarse to a fine grid of the same box: per
// axis, fine node i lies between coarse nodes lo[i] and lo[i] + 1 at fraction t[i]
// (lo = -1 and lo + 1 = n_c stand for the walls, where the Dirichlet value is 0).
struct InterpParams {
  int d;
  int nf[MAXD], nc[MAXD];
  long long cstride[MAXD];
  const int* lo[MAXD];
  const double* t[MAXD];
};

__global__ void k_interp(InterpParams ip, const double* __restrict__ uc, double* __restrict__ uf, long long Nf) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < Nf;
       idx += (long long)gridDim.x * blockDim.x) {
    int l[MAXD];
    double t[MAXD];
    long long q = idx;
    for (int k = 0; k < ip.d; ++k) {
      const long long qq = q / ip.nf[k];
      const int i = (int)(q - qq * ip.nf[k]);
      q = qq;
      l[k] = ip.lo[k][i];
      t[k] = ip.t[k][i];
    }
    double acc = 0.0;
    for (int corner = 0; corner < (1 << ip.d); ++corner) {
      double w = 1.0;
      long long off = 0;
      bool inside = true;
      for (int k = 0; k < ip.d; ++k) {
        const int b = (corner >> k) & 1;
        const int j = l[k] + b;
        w *= b ? t[k] : 1.0 - t[k];
        inside = inside && j >= 0 && j < ip.nc[k];
        off += (long long)j * ip.cstride[k];
      }
      if (inside && w != 0.0) acc = fma(w, uc[off], acc);
    }
    uf[idx] = acc;
  }
}

}  // namespace

int red_blocks() { return RED_BLOCKS; }

static inline unsigned grid_for(long long N) {
  long long g = (N + 255) / 256;
  return (unsigned)(g < RED_BLOCKS ? (g < 1 ? 1 : g) : RED_BLOCKS);
}

ts_status scale_inverse_fp64(const ts_plan* p, double sigma, double* X, cudaStream_t s) {
  k_scale_inverse<<<grid_for(p->N), 256, 0, s>>>(axis_params(p, true), sigma, X, p->N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status scale_exp_c128(const ts_plan* p, double tau, double* X, cudaStream_t s) {
  k_scale_exp<<<grid_for(p->N), 256, 0, s>>>(axis_params(p, true), tau, X, p->N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status phase_v2_c128(long long N, const double* V2, double th, double* psi, cudaStream_t s) {
  k_phase_c128<<<grid_for(N), 256, 0, s>>>(V2, th, psi, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status phase_v2_c64(long long N, const double* V2, double th, float* psi, cudaStream_t s) {
  k_phase_c64<<<grid_for(N), 256, 0, s>>>(V2, th, psi, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status convert_c64_to_c128(long long N, const float* in, double* out, cudaStream_t s) {
  k_c64_to_c128<<<grid_for(2 * N), 256, 0, s>>>(in, out, 2 * N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status convert_c128_to_c64(long long N, const double* in, float* out, cudaStream_t s) {
  k_c128_to_c64<<<grid_for(2 * N), 256, 0, s>>>(in, out, 2 * N);
  TS_LAUNCHED(1);
  return TS_OK;
}

namespace {
BandParams band_params(const ts_plan* p) {
  BandParams a{};
  a.d = p->d;
  a.order = p->order;
  long long st = 1;
  for (int k = 0; k < p->d; ++k) {
    a.w[k] = band_halfwidth(p, k);
    a.n[k] = p->n[k];
    a.stride[k] = st;
    st *= p->n[k];
    a.band[k] = p->band[k];
    a.f[k] = p->f[k];
  }
  return a;
}
}  // namespace

namespace {
WeightParams weight_params(const ts_plan* p) {
  WeightParams w{};
  w.d = p->d;
  for (int k = 0; k < p->d; ++k) {
    w.n[k] = p->n[k];
    w.mh[k] = p->order >= 2 ? p->mh[k] : nullptr;
    w.h[k] = 2.0 * p->L[k] / (p->n[k] + 1);
  }
  return w;
}
}  // namespace

ts_status wdot2(const ts_plan* p, const double* a, const double* b, const double* c, const double* d,
                double* partial, double* out2, cudaStream_t s) {
  k_wdot<0><<<RED_BLOCKS, 256, 0, s>>>(weight_params(p), a, b, c, d, p->N, partial);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, RED_BLOCKS, out2);
  TS_LAUNCHED(2);
  return TS_OK;
}

ts_status wdot_energy(const ts_plan* p, const double* u, const double* Hu, double* partial, double* out2,
                      cudaStream_t s) {
  k_wdot<1><<<RED_BLOCKS, 256, 0, s>>>(weight_params(p), u, Hu, nullptr, nullptr, p->N, partial);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, RED_BLOCKS, out2);
  TS_LAUNCHED(2);
  return TS_OK;
}

ts_status wdot_residual(const ts_plan* p, const double* u, const double* Hu, double lambda, double* partial,
                        double* out2, cudaStream_t s) {
  k_wdot<2><<<RED_BLOCKS, 256, 0, s>>>(weight_params(p), u, Hu, nullptr, nullptr, p->N, partial, lambda);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, RED_BLOCKS, out2);
  TS_LAUNCHED(2);
  return TS_OK;
}

ts_status gpe_veff(long long N, const double* V2, double beta, const double* u, double* veff, cudaStream_t s) {
  k_gpe_veff<<<grid_for(N), 256, 0, s>>>(V2, beta, u, veff, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status axpy2(long long N, double* u, double a, const double* x, double b, const double* y, cudaStream_t s) {
  k_axpy2<<<grid_for(N), 256, 0, s>>>(u, a, x, b, y, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status interpolate(const ts_plan* pc, const double* uc, const ts_plan* pf, double* uf, cudaStream_t s) {
  TS_REQUIRE(pc->d == pf->d, "interpolation needs grids of one dimension (%d, %d)", pc->d, pf->d);
  if (pc->order == -1 || pf->order == -1) {
    set_error("interpolation between grids of bounded boxes only (not Hermite grids on R^d)");
    return TS_ERR_UNSUPPORTED;
  }
  const int d = pc->d;
  for (int k = 0; k < d; ++k)
    TS_REQUIRE(pc->L[k] == pf->L[k], "interpolation needs the same box (axis %d: L = %g, %g)", k, pc->L[k], pf->L[k]);
  // per axis: coarse nodes with the two walls, and the bracket of every fine node
  std::vector<int> lo_h;
  std::vector<double> t_h;
  std::vector<size_t> off(d);
  for (int k = 0; k < d; ++k) {
    std::vector<double> xc(pc->n[k]), xf(pf->n[k]);
    TS_TRY(grid_nodes_host(pc->n[k], pc->L[k], pc->order, xc.data(), nullptr));
    TS_TRY(grid_nodes_host(pf->n[k], pf->L[k], pf->order, xf.data(), nullptr));
    std::vector<double> ext(pc->n[k] + 2);
    ext[0] = -pc->L[k];
    for (int i = 0; i < pc->n[k]; ++i) ext[i + 1] = xc[i];
    ext[pc->n[k] + 1] = pc->L[k];
    off[k] = lo_h.size();
    for (int i = 0; i < pf->n[k]; ++i) {
      const double x = xf[i];
      int j = (int)(std::upper_bound(ext.begin(), ext.end(), x) - ext.begin()) - 1;  // ext[j] <= x < ext[j+1]
      j = j < 0 ? 0 : (j > pc->n[k] ? pc->n[k] : j);
      lo_h.push_back(j - 1);
      t_h.push_back((x - ext[j]) / (ext[j + 1] - ext[j]));
    }
  }
  void* tab = nullptr;
  const size_t nl = lo_h.size();
  TS_TRY(scratch_alloc(&tab, sizeof(double) * nl + sizeof(int) * nl + 256, s));
  double* t_d = static_cast<double*>(tab);
  int* lo_d = reinterpret_cast<int*>(t_d + nl);
  ts_status st = TS_OK;
  if (cudaMemcpyAsync(t_d, t_h.data(), sizeof(double) * nl, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(lo_d, lo_h.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("interpolation tables: copy failed");
    st = TS_ERR_CUDA;
  }
  if (st == TS_OK) {
    InterpParams ip{};
    ip.d = d;
    long long cs = 1;
    for (int k = 0; k < d; ++k) {
      ip.nf[k] = pf->n[k];
      ip.nc[k] = pc->n[k];
      ip.cstride[k] = cs;
      cs *= pc->n[k];
      ip.lo[k] = lo_d + off[k];
      ip.t[k] = t_d + off[k];
    }
    k_interp<<<grid_for(pf->N), 256, 0, s>>>(ip, uc, uf, pf->N);
    TS_LAUNCHED(1);
    // the host vectors go out of scope: wait for the copies
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("interpolation failed");
      st = TS_ERR_CUDA;
    }
  }
  scratch_free(tab, s);
  return st;
}

ts_status scale_separable(const ts_plan* p, bool inverse, const double* x, double* y, cudaStream_t s) {
  AxisParams a = axis_params(p, false);
  for (int k = 0; k < p->d; ++k) a.tab[k] = inverse ? p->mhi[k] : p->mh[k];
  k_scale_separable<<<grid_for(p->N), 256, 0, s>>>(a, x, y, p->N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status stencil_apply(const ts_plan* p, const double* V2, double sigma, const double* x, double* y,
                        double* partial, double* out2, cudaStream_t s) {
  unsigned g = grid_for(p->N);
  if (banded_plan(p))
    k_banded<0, 2><<<g, 256, 0, s>>>(band_params(p), V2, sigma, x, nullptr, y, nullptr, p->N, partial);
  else
  k_stencil<0, 2><<<g, 256, 0, s>>>(axis_params(p, false), V2, sigma, x, nullptr, y, nullptr, p->N, partial);
  TS_LAUNCHED(1);
  if (out2) {
    k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)g, out2);
    TS_LAUNCHED(1);
  }
  return TS_OK;
}

ts_status stencil_residual(const ts_plan* p, const double* V2, double sigma, const double* x, const double* b,
                           double* r, double* partial, double* out2, cudaStream_t s) {
  unsigned g = grid_for(p->N);
  if (banded_plan(p))
    k_banded<1, 2><<<g, 256, 0, s>>>(band_params(p), V2, sigma, x, b, r, nullptr, p->N, partial);
  else
    k_stencil<1, 2><<<g, 256, 0, s>>>(axis_params(p, false), V2, sigma, x, b, r, nullptr, p->N, partial);
  TS_LAUNCHED(1);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)g, out2);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status stencil_residual_split(const ts_plan* p, const double* V2, double sigma, const double* x,
                                 const double* b, __nv_bfloat16* planes, int np, double* partial, cudaStream_t s) {
  unsigned g = grid_for(p->N);
  if (banded_plan(p)) {
    const BandParams a = band_params(p);
    if (np == 1)
      k_banded<2, 1><<<g, 256, 0, s>>>(a, V2, sigma, x, b, nullptr, planes, p->N, partial);
    else if (np == 2)
      k_banded<2, 2><<<g, 256, 0, s>>>(a, V2, sigma, x, b, nullptr, planes, p->N, partial);
    else
      k_banded<2, 3><<<g, 256, 0, s>>>(a, V2, sigma, x, b, nullptr, planes, p->N, partial);
  } else if (np == 1)
    k_stencil<2, 1><<<g, 256, 0, s>>>(axis_params(p, false), V2, sigma, x, b, nullptr, planes, p->N, partial);
  else if (np == 2)
    k_stencil<2, 2><<<g, 256, 0, s>>>(axis_params(p, false), V2, sigma, x, b, nullptr, planes, p->N, partial);
  else
    k_stencil<2, 3><<<g, 256, 0, s>>>(axis_params(p, false), V2, sigma, x, b, nullptr, planes, p->N, partial);
  TS_LAUNCHED(1);
  return TS_OK;
}

bool isotropic_h(const ts_plan* p) {
  if (banded_plan(p)) return false;  // Q^k and Hermite nodes are not equally spaced
  for (int k = 1; k < p->d; ++k)
    if (2.0 * p->L[k] / (p->n[k] + 1) != 2.0 * p->L[0] / (p->n[0] + 1)) return false;
  return true;
}

int qtable_count(const ts_plan* p) { return p->d == 3 ? 1 + p->n[0] + p->n[1] + p->n[2] : 0; }

namespace {
ts_status residual_split_fixed_launch(const ts_plan* p, double sigma, const double* x, const double* b,
                                      __nv_bfloat16* planes, int np, const int* emax_dev, long long* qtab,
                                      cudaStream_t s);
}  // namespace

// Times the kernel (profiling kind PROF_RESIDUAL: x, b in, NP bf16 planes out).
ts_status residual_split_fixed(const ts_plan* p, double sigma, const double* x, const double* b,
                               __nv_bfloat16* planes, int np, const int* emax_dev, long long* qtab, cudaStream_t s) {
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  const ts_status st = residual_split_fixed_launch(p, sigma, x, b, planes, np, emax_dev, qtab, s);
  if (tok) prof_end_launch(s, tok, PROF_RESIDUAL, 0.0, (16.0 + 2.0 * np) * (double)p->N);
  return st;
}

namespace {
template <int NP, int P, bool QF, bool APPLY = false>
ts_status launch_march3(long long blocks, const AxisParams& a, double sigma, const long long* Q, int F,
                        const double* x, const double* b, __nv_bfloat16* planes, long long N, const int* emax_dev,
                        cudaStream_t s, double* yout = nullptr, double* partial = nullptr) {
  static bool attr_set = false;  // per instantiation: the ring is dynamic shared memory
  if (!attr_set) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_residual_march3<NP, P, QF, APPLY>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, RING_BYTES));
    attr_set = true;
  }
  k_residual_march3<NP, P, QF, APPLY>
      <<<(unsigned)blocks, 256, RING_BYTES, s>>>(a, sigma, Q, F, x, b, planes, N, emax_dev, yout, partial);
  return TS_OK;
}

// Fixed-point headroom H and fraction bits F of the folded diagonal for sigma + V1
// (d = 3, one spacing): q_max bounds |sigma + V1| / h^-2; H leaves room for
// (4d + q_max + 1) 2^H <= 2^62 and F for q_max 2^F < 2^62.  False when fewer than 53 bits
// of headroom would remain.
bool fold_params(const ts_plan* p, double sigma, int* Hq_out, int* F_out) {
  if (p->d != 3 || !isotropic_h(p)) return false;
  double fmax = std::fabs(sigma);
  for (int k = 0; k < 3; ++k) {
    double m = 0.0;
    for (double v : p->axis[k]->f) m = std::fmax(m, std::fabs(v));
    fmax += m;
  }
  const double h = 2.0 * p->L[0] / (p->n[0] + 1);
  const double qmax = fmax / (1.0 / (h * h));
  if (!std::isfinite(qmax)) return false;
  int Hq = 58;
  while (Hq >= 53 && std::ldexp(4.0 * p->d + qmax + 1.0, Hq) > std::ldexp(1.0, 62)) --Hq;
  int F = 62;
  while (F > Hq && std::ldexp(qmax + 1.0, F) >= std::ldexp(1.0, 62)) --F;
  *Hq_out = Hq;
  *F_out = F;
  return Hq >= 53 && F >= Hq;
}

long long march_blocks(const ts_plan* p) {
  return (long long)((p->n[0] + MX - 1) / MX) * ((p->n[1] + MY - 1) / MY) * ((p->n[2] + MZ - 1) / MZ);
}

ts_status residual_split_fixed_launch(const ts_plan* p, double sigma, const double* x, const double* b,
                                      __nv_bfloat16* planes, int np, const int* emax_dev, long long* qtab,
                                      cudaStream_t s) {
  int H = 62;  // headroom: 2d |U| + 2d |U| < 2^63
  for (long long t = 4LL * p->d; t > 1; t = (t + 1) / 2) --H;
  const AxisParams a = axis_params(p, false);
  if (p->d == 3) {
    const long long blocks = (long long)((p->n[0] + MX - 1) / MX) * ((p->n[1] + MY - 1) / MY) *
                             ((p->n[2] + MZ - 1) / MZ);
    int Hq = 0, F = 0;
    const bool fold = fold_params(p, sigma, &Hq, &F);
    if (qtab && fold) {
      const int total = qtable_count(p);
      k_qtables<<<(total + 127) / 128, 128, 0, s>>>(p->f[0], p->n[0], p->f[1], p->n[1], p->f[2], p->n[2], sigma,
                                                    a.ih2[0], F, qtab);
      TS_LAUNCHED(1);
#define TS_QF_CASE(PP)                                                                                  \
  case PP:                                                                                              \
    if (np == 1)                                                                                        \
      TS_TRY((launch_march3<1, PP, true>(blocks, a, sigma, qtab, F, x, b, planes, p->N, emax_dev, s)));  \
    else if (np == 2)                                                                                   \
      TS_TRY((launch_march3<2, PP, true>(blocks, a, sigma, qtab, F, x, b, planes, p->N, emax_dev, s)));  \
    else                                                                                                \
      TS_TRY((launch_march3<3, PP, true>(blocks, a, sigma, qtab, F, x, b, planes, p->N, emax_dev, s)));  \
    break;
      switch (Hq - 53) {
        TS_QF_CASE(0) TS_QF_CASE(1) TS_QF_CASE(2) TS_QF_CASE(3) TS_QF_CASE(4)
        default: TS_QF_CASE(5)
      }
#undef TS_QF_CASE
      TS_LAUNCHED(1);
      return TS_OK;
    }
    if (np == 1)
      TS_TRY((launch_march3<1, 5, false>(blocks, a, sigma, nullptr, 0, x, b, planes, p->N, emax_dev, s)));
    else if (np == 2)
      TS_TRY((launch_march3<2, 5, false>(blocks, a, sigma, nullptr, 0, x, b, planes, p->N, emax_dev, s)));
    else
      TS_TRY((launch_march3<3, 5, false>(blocks, a, sigma, nullptr, 0, x, b, planes, p->N, emax_dev, s)));
    TS_LAUNCHED(1);
    return TS_OK;
  }
  if (np == 1)
    k_residual_fixed<1><<<grid_for(p->N), 256, 0, s>>>(a, sigma, x, b, planes, p->N, emax_dev, H);
  else if (np == 2)
    k_residual_fixed<2><<<grid_for(p->N), 256, 0, s>>>(a, sigma, x, b, planes, p->N, emax_dev, H);
  else
    k_residual_fixed<3><<<grid_for(p->N), 256, 0, s>>>(a, sigma, x, b, planes, p->N, emax_dev, H);
  TS_LAUNCHED(1);
  return TS_OK;
}
}  // namespace

namespace {
// Largest biased exponent over x (integer max of the exponent bits; order-independent).
__global__ void k_max_exponent(const double* __restrict__ x, long long N, int* out) {
  int m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (__double2hiint(x[i]) >> 20) & 0x7FF);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
}  // namespace

ts_status max_exponent(const double* x, long long N, int* emax, cudaStream_t s) {
  TS_CHECK_CUDA(cudaMemsetAsync(emax, 0, sizeof(int), s));
  k_max_exponent<<<grid_for(N), 256, 0, s>>>(x, N, emax);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status residual_fixed(const ts_plan* p, const FixedOperator& fo, const double* V2, const double* x,
                         const double* b, double* r, int* emax, double* opart, double* partial, double* out2,
                         cudaStream_t s) {
  TS_TRY(max_exponent(x, p->N, emax, s));
  TS_TRY(operator_apply_fixed(p, fo, V2, x, r, emax, opart, nullptr, s));  // r = A x
  const unsigned g = grid_for(p->N);
  k_sub_dot<<<g, 256, 0, s>>>(b, r, p->N, partial);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)g, out2);
  TS_LAUNCHED(2);
  return TS_OK;
}

ts_status operator_apply(const ts_plan* p, const double* V2, double sigma, const double* x, double* y,
                         cudaStream_t s) {
  int H = 0, F = 0;
  if (!fold_params(p, sigma, &H, &F)) {
    void* partial = nullptr;
    TS_TRY(scratch_alloc(&partial, sizeof(double) * 2 * RED_BLOCKS, s));
    const ts_status st = stencil_apply(p, V2, sigma, x, y, (double*)partial, nullptr, s);
    scratch_free(partial, s);
    return st;
  }
  const long long blocks = march_blocks(p);
  // one allocation: the exponent, the Q tables, the per-block partials
  const size_t qbytes = sizeof(long long) * (size_t)qtable_count(p);
  void* work = nullptr;
  TS_TRY(scratch_alloc(&work, 256 + qbytes + sizeof(double) * 2 * (size_t)blocks, s));
  char* w = static_cast<char*>(work);
  int* emax = reinterpret_cast<int*>(w);
  long long* qtab = reinterpret_cast<long long*>(w + 256);
  double* partial = reinterpret_cast<double*>(w + 256 + qbytes);
  ts_status st = TS_OK;
  if (cudaMemsetAsync(emax, 0, sizeof(int), s) != cudaSuccess) {
    set_error("memset failed");
    st = TS_ERR_CUDA;
  }
  if (st == TS_OK) {
    k_max_exponent<<<grid_for(p->N), 256, 0, s>>>(x, p->N, emax);
    count_launches(1);
    FixedOperator fo;
    st = fixed_operator_prepare(p, sigma, qtab, &fo, s);
    if (st == TS_OK) st = operator_apply_fixed(p, fo, V2, x, y, emax, partial, nullptr, s);
  }
  scratch_free(work, s);
  return st;
}

ts_status fixed_operator_prepare(const ts_plan* p, double sigma, long long* qtab, FixedOperator* fo,
                                 cudaStream_t s) {
  fo->ok = false;
  if (!fold_params(p, sigma, &fo->H, &fo->F)) return TS_OK;
  const AxisParams a = axis_params(p, false);
  const int total = qtable_count(p);
  k_qtables<<<(total + 127) / 128, 128, 0, s>>>(p->f[0], p->n[0], p->f[1], p->n[1], p->f[2], p->n[2], sigma,
                                                a.ih2[0], fo->F, qtab);
  TS_LAUNCHED(1);
  fo->qtab = qtab;
  fo->sigma = sigma;
  fo->blocks = march_blocks(p);
  fo->ok = true;
  return TS_OK;
}

ts_status operator_apply_fixed(const ts_plan* p, const FixedOperator& fo, const double* V2, const double* x, double* y,
                               const int* emax_dev, double* partial, double* out2, cudaStream_t s) {
  const AxisParams a = axis_params(p, false);
#define TS_OP_CASE(PP)                                                                                     \
  case PP:                                                                                                 \
    TS_TRY((launch_march3<1, PP, true, true>(fo.blocks, a, fo.sigma, fo.qtab, fo.F, x, V2, nullptr, p->N, emax_dev, \
                                             s, y, partial)));                                             \
    break;
  switch (fo.H - 53) {
    TS_OP_CASE(0) TS_OP_CASE(1) TS_OP_CASE(2) TS_OP_CASE(3) TS_OP_CASE(4)
    default: TS_OP_CASE(5)
  }
#undef TS_OP_CASE
  TS_LAUNCHED(1);
  if (out2) {
    k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)fo.blocks, out2);
    TS_LAUNCHED(1);
  }
  return TS_OK;
}

ts_status dot2(long long N, const double* a, const double* b, const double* c, const double* d, double* partial,
               double* out2, cudaStream_t s) {
  unsigned g = grid_for(N);
  k_dot2<<<g, 256, 0, s>>>(a, b, c, d, N, partial);
  TS_LAUNCHED(1);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)g, out2);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status pcg_update_xr(const double* rz, const double* pq, double* alpha_out, double* x, double* r,
                        const double* p, const double* q, long long N, double* partial, double* out2,
                        cudaStream_t s) {
  unsigned g = grid_for(N);
  k_pcg_xr<<<g, 256, 0, s>>>(rz, pq, alpha_out, x, r, p, q, N, partial);
  TS_LAUNCHED(1);
  k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)g, out2);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status pcg_update_p(const double* alpha, const double* zq, const double* rz_old, int first, double* p,
                       const double* z, long long N, cudaStream_t s, int* emax_out) {
  if (emax_out) TS_CHECK_CUDA(cudaMemsetAsync(emax_out, 0, sizeof(int), s));
  k_pcg_p<<<grid_for(N), 256, 0, s>>>(alpha, zq, rz_old, first, p, z, N, emax_out);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status copy_scalar(const double* src, double* dst, cudaStream_t s) {
  k_copy_scalar<<<1, 1, 0, s>>>(src, dst);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status tensor_ground(const ts_plan* p, double* u, cudaStream_t s) {
  AxisParams a = axis_params(p, true);
  for (int k = 0; k < p->d; ++k) a.tab[k] = p->St[k];
  k_tensor_ground<<<grid_for(p->N), 256, 0, s>>>(a, u, p->N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status axpby(long long N, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<grid_for(N), 256, 0, s>>>(a, x, b, y, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status scale_by_device_ratio(long long N, const double* num, const double* den, const double* x, double* y,
                                cudaStream_t s) {
  k_scale_by_scalar<<<grid_for(N), 256, 0, s>>>(num, den, y, x, N);
  TS_LAUNCHED(1);
  return TS_OK;
}

}  // namespace ts
