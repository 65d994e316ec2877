// Fused multi-mode propagation for small axis lengths (n <= 32), complex64 data, FP32
// arithmetic: the exact propagator e^{-i tau (-Delta + V1)} (eq. exact_prop) of the 4D-9D
// problems, and the Strang step (Sec. 5.1) with the e^{-i V2 theta} factors folded into
// the first and last pass.
//
// -Delta_h + V1 = sum_k H_k with H_k acting on axis k alone, so the exact propagator is the
// tensor product of per-axis propagators: e^{-i tau (-Delta_h + V1)} = kron_k E_k with
// E_k = T_k diag(e^{-i tau lambda_k}) T_k^{-1} (steps 2-4 of Sec. 2.1 on one axis, an n x n
// complex matrix formed once per call in FP64).  Applying E_k directly costs the same FFMA as
// the forward transform, the phase and the backward transform along the axis, but leaves no
// intermediate in the eigenbasis: a step is ceil(d / f) HBM passes for groups of f axes,
// where the forward / phase / backward form needs 2 ceil(d / f) - 1.
//
// Axes are cut into groups of consecutive modes.  For a group [k0, k1) with
// lo = prod_{j<k0} n_j, G = prod_{k0<=j<k1} n_j and hi = prod_{j>=k1} n_j, a CTA owns the
// tile of T consecutive lo-indices (or, for k0 = 0, T consecutive hi-indices) times all G
// group indices: runs of >= 8 contiguous elements in HBM, so loads and stores coalesce.
// Input and output may be the same array: a CTA reads its whole tile before writing it.
// CTAs are persistent over tiles and double-buffer them: while one tile is contracted the
// next one arrives by cp.async.  In shared memory every group extent is padded to an odd
// length, so that the fibers of any mode start on distinct banks.  Each mode is applied by
// per-thread fibers held in registers (n complex values in, n out, 4 n^2 FFMA per fiber)
// with the matrix read from shared memory as broadcasts, in place.  The group shape (n and
// the number of modes) is a template parameter, so every index computation is by constants.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "async_copy.cuh"
#include "small_n.cuh"

namespace ts {
namespace {

constexpr int MAXG = 3;                     // modes per group
constexpr size_t TILE_BUDGET = 48 * 1024;   // bytes of one complex64 tile buffer (two per CTA)

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Threads per CTA: the 24-point groups hold 8 x 24 fibers per mode (T = 8), so 192 threads
// take one each with 170 registers at two CTAs per SM; the others use 256.
template <int N>
struct SmallCfg {
  static constexpr int THREADS = N == 24 ? 192 : 256;
  static constexpr int FPT = N <= 8 ? 2 : 1;  // fibers per thread sharing every matrix load
};

struct PropParams {
  long long lo, hi;         // extents below / above the group
  int T;                    // tile count along lo (lo > 1) or along hi (lo == 1), a power of two
  const float2* E[MAXG];    // per mode of the group: ET[i'][i] = E_k[i][i'] (n x n, complex)
  // potential phase e^{-i theta V2}: applied on load (theta_pre) / on store (theta_post)
  const float* V2;
  float theta_pre, theta_post;
  // Element pairs in the copies between HBM and the tile (index arithmetic once per pair):
  // 1: lo > 1 with an even tile count T and 16-byte aligned X and Y, so elements (t, t + 1)
  //    for even t are adjacent in HBM and in shared memory: one 16-byte copy each way;
  // 2: lo == 1 with an even first extent and 16-byte aligned Y: elements (i, i + 1) of the
  //    first group axis, i even, are adjacent in HBM and in shared memory, where the padded
  //    rows leave them 8-byte aligned: two 8-byte copies in, one 16-byte store out;
  // 0: one element at a time.
  int pairs;
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 vphase(float2 v, float theta, float V) {
  float s, c;
  __sincosf(theta * V, &s, &c);
  return cmulf(v, make_float2(c, -s));
}

// Padded offset of the group-flattened index g (D base-N digits, fastest first) in a tile
// whose extents are padded to N | 1.
template <int N, int D>
__device__ __forceinline__ int padded_offset(int g) {
  int r = 0;
#pragma unroll
  for (int k = 0, mul = 1; k < D; ++k, mul *= (N | 1)) {
    const int q = g / N;
    r += (g - q * N) * mul;
    g = q;
  }
  return r;
}

// Apply the matrix of mode M of the group, y_i = sum_i' E[i][i'] x_i' (Em holds ET[i'][i]),
// along every fiber of that mode of the tile, in place.  FPT fibers per thread and step
// (fibers f and f + THREADS) share every matrix load from shared memory; the output blocks
// are a rolled loop, so that the code of a mode stays small.
template <int N, int NM, int M, int FPT>
__device__ __forceinline__ void prop_mode(float2* tile, const float2* Em, int lgTlo, int Thi) {
  constexpr int THREADS = SmallCfg<N>::THREADS;
  constexpr int NPD = N | 1;
  constexpr int INNER_G = ipow(N, M), OUTER_G = ipow(N, NM - 1 - M);
  constexpr int STRIDE_G = ipow(NPD, M);  // padded stride of mode M (times Tlo)
  constexpr int GP = ipow(NPD, NM);
  constexpr int JB = N >= 16 ? 4 : 8;     // outputs per accumulation block
  static_assert(N % JB == 0, "axis length must be a multiple of the output block");
  const int Tlo = 1 << lgTlo;
  const int st = Tlo * STRIDE_G;
  const int fibers = Tlo * INNER_G * OUTER_G * Thi;
  for (int f0 = threadIdx.x; f0 < fibers; f0 += FPT * THREADS) {
    int addr[FPT];
    float2 x[FPT][N];
#pragma unroll
    for (int c = 0; c < FPT; ++c) {
      const int f = f0 + c * THREADS < fibers ? f0 + c * THREADS : f0;  // a missing partner repeats f0
      const int t = f & (Tlo - 1);
      int r = f >> lgTlo;
      const int gi = r % INNER_G;
      r /= INNER_G;
      const int go = r % OUTER_G;
      const int th = r / OUTER_G;
      addr[c] = t + Tlo * (padded_offset<N, M>(gi) + STRIDE_G * NPD * padded_offset<N, NM - 1 - M>(go) + GP * th);
#pragma unroll
      for (int i = 0; i < N; ++i) x[c][i] = tile[addr[c] + i * st];
    }
    const bool second = FPT > 1 && f0 + THREADS < fibers;
#pragma unroll 1
    for (int j0 = 0; j0 < N; j0 += JB) {
      float re[FPT][JB], im[FPT][JB];
#pragma unroll
      for (int c = 0; c < FPT; ++c)
#pragma unroll
        for (int q = 0; q < JB; ++q) re[c][q] = im[c][q] = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int q = 0; q < JB; q += 2) {
          const float4 e = *reinterpret_cast<const float4*>(Em + i * N + j0 + q);  // E[j0+q][i], E[j0+q+1][i]
#pragma unroll
          for (int c = 0; c < FPT; ++c) {
            re[c][q] = fmaf(e.x, x[c][i].x, re[c][q]);
            re[c][q] = fmaf(-e.y, x[c][i].y, re[c][q]);
            im[c][q] = fmaf(e.x, x[c][i].y, im[c][q]);
            im[c][q] = fmaf(e.y, x[c][i].x, im[c][q]);
            re[c][q + 1] = fmaf(e.z, x[c][i].x, re[c][q + 1]);
            re[c][q + 1] = fmaf(-e.w, x[c][i].y, re[c][q + 1]);
            im[c][q + 1] = fmaf(e.z, x[c][i].y, im[c][q + 1]);
            im[c][q + 1] = fmaf(e.w, x[c][i].x, im[c][q + 1]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < JB; ++q) {
        tile[addr[0] + (j0 + q) * st] = make_float2(re[0][q], im[0][q]);
        if (FPT > 1 && second) tile[addr[FPT - 1] + (j0 + q) * st] = make_float2(re[FPT - 1][q], im[FPT - 1][q]);
      }
    }
  }
}

template <int N, int NM, int M>
__device__ __forceinline__ void prop_modes(float2* tile, const float2* E, int lgTlo, int Thi) {
  if constexpr (M < NM) {
    prop_mode<N, NM, M, SmallCfg<N>::FPT>(tile, E + M * N * N, lgTlo, Thi);
    __syncthreads();
    prop_modes<N, NM, M + 1>(tile, E, lgTlo, Thi);
  }
}

// Shared-memory offset and group-flattened index of tile element e (global order: t
// fastest, then the group indices, then th).
template <int N, int NM>
__device__ __forceinline__ int tile_offset(int e, int lgTlo, int* g_out, int* th_out) {
  constexpr int G = ipow(N, NM), GP = ipow(N | 1, NM);
  const int t = e & ((1 << lgTlo) - 1);
  const int r = e >> lgTlo;
  const int g = r % G, th = r / G;
  *g_out = g;
  *th_out = th;
  return t + ((padded_offset<N, NM>(g) + GP * th) << lgTlo);
}

// Persistent over tiles with two shared-memory tile buffers: the next tile's elements are
// copied asynchronously (cp.async into the padded layout) while the current tile is
// contracted, so global-load latency overlaps arithmetic.
template <int N, int NM>
__global__ void __launch_bounds__(SmallCfg<N>::THREADS, 2) k_small_prop(const float2* X, float2* Y,
                                                                     const PropParams p, long long ntiles) {
  constexpr int SMALL_THREADS = SmallCfg<N>::THREADS;
  constexpr int G = ipow(N, NM), GP = ipow(N | 1, NM);
  extern __shared__ __align__(16) float2 smem[];
  const int lgT = 31 - __clz(p.T);
  const int lgTlo = p.lo > 1 ? lgT : 0;
  const int Tlo = 1 << lgTlo;
  const int Thi = p.lo > 1 ? 1 : p.T;
  const int tile_stride = (Tlo * GP * Thi + 1) & ~1;  // keep every buffer 16-byte aligned
  float2* buf[2] = {smem, smem + tile_stride};
  float2* mats = smem + 2 * tile_stride;
  for (int e = threadIdx.x; e < NM * N * N; e += SMALL_THREADS) mats[e] = p.E[e / (N * N)][e % (N * N)];
  const int cnt = Tlo * G * Thi;
  const long long loG = p.lo * G;
  auto origin = [&](long long b) -> long long {  // HBM index of the tile's first element
    if (p.lo > 1) {
      const long long lblocks = p.lo >> lgTlo;
      return ((b % lblocks) << lgTlo) + loG * (b / lblocks);
    }
    return loG * b * Thi;
  };
  auto issue_load = [&](long long b, float2* dst) {
    const long long gbase = origin(b);
    if (p.pairs == 1) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        cp_async16(dst + sidx, X + gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th));
      }
    } else if (p.pairs == 2) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const float2* src = X + gbase + p.lo * ((long long)g + (long long)G * th);
        cp_async8(dst + sidx, src);
        cp_async8(dst + sidx + 1, src + 1);
      }
    } else {
      for (int e = threadIdx.x; e < cnt; e += SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        cp_async8(dst + sidx, X + gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th));
      }
    }
    cp_async_commit();
  };
  long long b = blockIdx.x;
  if (b < ntiles) issue_load(b, buf[0]);
  int cur = 0;
  const int step_e = p.pairs ? 2 : 1;  // both pair kinds: (e, e + 1) at (sidx, sidx + 1)
  for (; b < ntiles; b += gridDim.x, cur ^= 1) {
    const long long bn = b + gridDim.x;
    if (bn < ntiles) {
      issue_load(bn, buf[cur ^ 1]);
      cp_async_wait<1>();  // the current tile's group has landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float2* tile = buf[cur];
    const long long gbase = origin(b);
    if (p.V2 && p.theta_pre != 0.f) {
      for (int e = step_e * threadIdx.x; e < cnt; e += step_e * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        tile[sidx] = vphase(tile[sidx], p.theta_pre, p.V2[gidx]);
        if (p.pairs) tile[sidx + 1] = vphase(tile[sidx + 1], p.theta_pre, p.V2[gidx + 1]);
      }
      __syncthreads();
    }
    prop_modes<N, NM, 0>(tile, mats, lgTlo, Thi);
    if (p.pairs) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        float2 v0 = tile[sidx], v1 = tile[sidx + 1];
        if (p.V2 && p.theta_post != 0.f) {
          v0 = vphase(v0, p.theta_post, p.V2[gidx]);
          v1 = vphase(v1, p.theta_post, p.V2[gidx + 1]);
        }
        *reinterpret_cast<float4*>(Y + gidx) = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    } else {
      for (int e = threadIdx.x; e < cnt; e += SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        float2 v = tile[sidx];
        if (p.V2 && p.theta_post != 0.f) v = vphase(v, p.theta_post, p.V2[gidx]);
        Y[gidx] = v;
      }
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
}

// 8-point axes in groups of three with T = 8: the tile is eight independent 8 x 8 x 8 cubes
// (one per lo index t, or per hi index th), and warp w owns cube w.  A warp applies its
// cube's three axis propagators alone (two fibers per lane sharing every matrix load),
// separated by __syncwarp instead of CTA barriers; only the copies between HBM and the
// tile are cooperative (64-byte runs along t for lo > 1).  Cube c starts at c * CUBE in
// shared memory, element (i0, i1, i2) at i0 + 9 i1 + 81 i2 (padded extents, odd).
constexpr int CUBE = 729;

template <int M>
__device__ __forceinline__ void cube_mode(float2* cube, const float2* Em, int lane) {
  // fibers of mode M: 64, indexed by the two other axes (the lower one fastest)
  constexpr int ST = M == 0 ? 1 : (M == 1 ? 9 : 81);
  constexpr int SA = M == 0 ? 9 : 1;   // stride of the fiber index's fast axis
  constexpr int SB = M == 2 ? 9 : 81;  // ... and of its slow axis
  int addr[2];
  float2 x[2][8];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int f = lane + 32 * c;
    addr[c] = (f & 7) * SA + (f >> 3) * SB;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[c][i] = cube[addr[c] + i * ST];
  }
  float re[2][8], im[2][8];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int q = 0; q < 8; ++q) re[c][q] = im[c][q] = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const float4 e = *reinterpret_cast<const float4*>(Em + i * 8 + q);  // E[q][i], E[q+1][i]
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        re[c][q] = fmaf(e.x, x[c][i].x, re[c][q]);
        re[c][q] = fmaf(-e.y, x[c][i].y, re[c][q]);
        im[c][q] = fmaf(e.x, x[c][i].y, im[c][q]);
        im[c][q] = fmaf(e.y, x[c][i].x, im[c][q]);
        re[c][q + 1] = fmaf(e.z, x[c][i].x, re[c][q + 1]);
        re[c][q + 1] = fmaf(-e.w, x[c][i].y, re[c][q + 1]);
        im[c][q + 1] = fmaf(e.z, x[c][i].y, im[c][q + 1]);
        im[c][q + 1] = fmaf(e.w, x[c][i].x, im[c][q + 1]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int q = 0; q < 8; ++q) cube[addr[c] + q * ST] = make_float2(re[c][q], im[c][q]);
}

__global__ void __launch_bounds__(256, 2) k_small_cubes(const float2* X, float2* Y, const PropParams p,
                                                       long long ntiles) {
  constexpr int TSZ = 8 * CUBE;  // one tile buffer
  extern __shared__ __align__(16) float2 smem[];
  float2* buf[2] = {smem, smem + TSZ};
  float2* mats = smem + 2 * TSZ;
  for (int e = threadIdx.x; e < 3 * 64; e += 256) mats[e] = p.E[e / 64][e % 64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool lo_tiles = p.lo > 1;  // cubes along lo (t = cube) or along hi (th = cube)
  auto origin = [&](long long b) -> long long {
    if (lo_tiles) {
      const long long lblocks = p.lo >> 3;
      return ((b % lblocks) << 3) + p.lo * 512 * (b / lblocks);
    }
    return 512LL * 8 * b;
  };
  // element e of a tile in HBM order (lo tiles: t fastest, then g; hi tiles: g fastest, then th)
  auto offsets = [&](int e, long long gbase, int* sidx, long long* gidx) {
    int c, g;
    if (lo_tiles) {
      c = e & 7;
      g = e >> 3;
      *gidx = gbase + c + p.lo * g;
    } else {
      c = e >> 9;
      g = e & 511;
      *gidx = gbase + e;
    }
    *sidx = c * CUBE + (g & 7) + 9 * ((g >> 3) & 7) + 81 * (g >> 6);
  };
  auto issue_load = [&](long long b, float2* dst) {
    const long long gbase = origin(b);
    if (p.pairs) {
      for (int e = 2 * threadIdx.x; e < 4096; e += 512) {
        int sidx;
        long long gidx;
        offsets(e, gbase, &sidx, &gidx);
        // lo tiles: (t, t + 1) are cubes t and t + 1; hi tiles: (i0, i0 + 1) of one cube row
        cp_async8(dst + sidx, X + gidx);
        cp_async8(dst + sidx + (lo_tiles ? CUBE : 1), X + gidx + 1);
      }
    } else {
      for (int e = threadIdx.x; e < 4096; e += 256) {
        int sidx;
        long long gidx;
        offsets(e, gbase, &sidx, &gidx);
        cp_async8(dst + sidx, X + gidx);
      }
    }
    cp_async_commit();
  };
  long long b = blockIdx.x;
  if (b < ntiles) issue_load(b, buf[0]);
  int cur = 0;
  for (; b < ntiles; b += gridDim.x, cur ^= 1) {
    const long long bn = b + gridDim.x;
    if (bn < ntiles) {
      issue_load(bn, buf[cur ^ 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // the tile has landed (copied by every thread)
    float2* cube = buf[cur] + warp * CUBE;
    const long long gbase = origin(b);
    if (p.V2 && p.theta_pre != 0.f) {
      // the warp's own cube: element g of cube `warp`
      for (int g = lane; g < 512; g += 32) {
        const long long gidx = lo_tiles ? gbase + warp + p.lo * g : gbase + 512LL * warp + g;
        const int si = (g & 7) + 9 * ((g >> 3) & 7) + 81 * (g >> 6);
        cube[si] = vphase(cube[si], p.theta_pre, p.V2[gidx]);
      }
      __syncwarp();
    }
    cube_mode<0>(cube, mats, lane);
    __syncwarp();
    cube_mode<1>(cube, mats + 64, lane);
    __syncwarp();
    cube_mode<2>(cube, mats + 128, lane);
    __syncthreads();  // every cube is done before the cooperative store
    float2* tile = buf[cur];
    const int step_e = p.pairs ? 2 : 1;
    for (int e = step_e * threadIdx.x; e < 4096; e += step_e * 256) {
      int sidx;
      long long gidx;
      offsets(e, gbase, &sidx, &gidx);
      float2 v0 = tile[sidx];
      if (p.pairs) {
        float2 v1 = tile[sidx + (lo_tiles ? CUBE : 1)];
        if (p.V2 && p.theta_post != 0.f) {
          v0 = vphase(v0, p.theta_post, p.V2[gidx]);
          v1 = vphase(v1, p.theta_post, p.V2[gidx + 1]);
        }
        *reinterpret_cast<float4*>(Y + gidx) = make_float4(v0.x, v0.y, v1.x, v1.y);
      } else {
        if (p.V2 && p.theta_post != 0.f) v0 = vphase(v0, p.theta_post, p.V2[gidx]);
        Y[gidx] = v0;
      }
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
}

ts_status launch_cubes(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s);

// ET[k][i'][i] = E_k[i][i'] with E_k[i][i'] = sum_l St[l][i] e^{-i tau lambda_l} S[i'][l]
// (FP64, rounded to FP32): the axis propagator T diag(e^{-i tau lambda}) T^{-1} in the plan's
// operands (forward y_l = sum_i' S[i'][l] x_i', backward y_i = sum_l St[l][i] x_l).
struct AxisOps {
  const double* S[MAXD];
  const double* St[MAXD];
  const double* lam[MAXD];
  int n[MAXD];
  int off[MAXD];  // offset of axis k's matrix in ET (elements)
};

__global__ void k_axis_propagators(const AxisOps a, int d, double tau, float2* ET) {
  const int k = blockIdx.y;
  if (k >= d) return;
  const int n = a.n[k];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int ip = e / n, i = e - ip * n;  // ET[i'][i]
  double re = 0.0, im = 0.0;
  for (int l = 0; l < n; ++l) {
    double s, c;
    sincos(tau * a.lam[k][l], &s, &c);
    const double w = a.St[k][(long long)l * n + i] * a.S[k][(long long)ip * n + l];
    re += w * c;
    im -= w * s;
  }
  ET[a.off[k] + e] = make_float2((float)re, (float)im);
}

__global__ void k_to_f32(const double* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void k_to_f32_table(const double* S, const double* St, float* Sf, float* Stf, int cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) {
    Sf[i] = (float)S[i];
    Stf[i] = (float)St[i];
  }
}

int odd(int n) { return n | 1; }

struct Group {
  int k0, k1, T;
};

// Groups of consecutive axes of equal length: each run of r axes of one length n is cut into
// ceil(r / f) groups of balanced sizes, f = the most modes whose padded tile (with T = 8,
// i.e. 64-byte runs) fits the budget.
std::vector<Group> make_groups(const ts_plan* p) {
  std::vector<std::pair<int, int>> spans;  // [k, k1) of the groups
  for (int a = 0; a < p->d;) {
    int b = a + 1;
    while (b < p->d && p->n[b] == p->n[a]) ++b;
    int f = 1;
    while (f < MAXG && f < b - a && (size_t)ipow(odd(p->n[a]), f + 1) * 8 * sizeof(float2) <= TILE_BUDGET) ++f;
    const int r = b - a, ng = (r + f - 1) / f;
    for (int g = 0, k = a; g < ng; ++g) {
      const int size = r / ng + (g < r % ng ? 1 : 0);
      spans.push_back({k, k + size});
      k += size;
    }
    a = b;
  }
  std::vector<Group> gs;
  for (const auto& sp : spans) {
    const int k = sp.first, k1 = sp.second;
    long long lo = 1, hi = 1, gpad = 1;
    for (int j = 0; j < k; ++j) lo *= p->n[j];
    for (int j = k1; j < p->d; ++j) hi *= p->n[j];
    for (int j = k; j < k1; ++j) gpad *= odd(p->n[j]);
    const long long along = lo > 1 ? lo : hi;
    int T = 1;
    while ((size_t)(gpad * (T * 2) * sizeof(float2)) <= TILE_BUDGET && along % (T * 2) == 0 && T < 256) T *= 2;
    gs.push_back({k, k1, T});
  }
  return gs;
}

int g_small_sms = 0;

template <int N, int NM>
ts_status launch_prop(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  constexpr int GP = ipow(N | 1, NM);
  const int Tlo = gp.lo > 1 ? gp.T : 1, Thi = gp.lo > 1 ? 1 : gp.T;
  const size_t tile_stride = ((size_t)Tlo * GP * Thi + 1) & ~size_t(1);
  const size_t smem = sizeof(float2) * (2 * tile_stride + (size_t)NM * N * N);
  static bool attr = false;
  if (!attr) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_prop<N, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  if (g_small_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_small_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long tiles = gp.lo > 1 ? (gp.lo / Tlo) * gp.hi : gp.hi / Thi;
  int per_sm = 0;
  constexpr int THREADS = SmallCfg<N>::THREADS;
  TS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_prop<N, NM>, THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  const long long grid = tiles < (long long)g_small_sms * per_sm ? tiles : (long long)g_small_sms * per_sm;
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_small_prop<N, NM><<<(unsigned)grid, THREADS, smem, s>>>(X, Y, gp, tiles);
  TS_LAUNCHED(1);
  if (tok) {
    const long long N_all = gp.lo * (long long)ipow(N, NM) * gp.hi;
    prof_end_launch(s, tok, PROF_SMALL_PASS, 8.0 * N * (double)N_all * NM, 16.0 * (double)N_all);
  }
  return TS_OK;
}

ts_status launch_cubes(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (2 * 8 * CUBE + 3 * 64);
  static bool attr = false;
  if (!attr) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_cubes, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  if (g_small_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_small_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long tiles = gp.lo > 1 ? (gp.lo / 8) * gp.hi : gp.hi / 8;
  int per_sm = 0;
  TS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_cubes, 256, smem));
  if (per_sm < 1) per_sm = 1;
  const long long grid = tiles < (long long)g_small_sms * per_sm ? tiles : (long long)g_small_sms * per_sm;
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_small_cubes<<<(unsigned)grid, 256, smem, s>>>(X, Y, gp, tiles);
  TS_LAUNCHED(1);
  if (tok) {
    const long long N_all = gp.lo * 512LL * gp.hi;
    prof_end_launch(s, tok, PROF_SMALL_PASS, 8.0 * 8 * (double)N_all * 3, 16.0 * (double)N_all);
  }
  return TS_OK;
}

ts_status group_pass(int n, int nm, const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  if (n == 8 && nm == 3 && gp.T == 8) return launch_cubes(X, Y, gp, s);  // one cube per warp
#define TS_PROP_CASE(NN)                                          \
  case NN:                                                        \
    if (nm == 1) return launch_prop<NN, 1>(X, Y, gp, s);          \
    if (nm == 2) return launch_prop<NN, 2>(X, Y, gp, s);          \
    return launch_prop<NN, 3>(X, Y, gp, s);
  switch (n) {
    TS_PROP_CASE(8)
    TS_PROP_CASE(16)
    TS_PROP_CASE(24)
    TS_PROP_CASE(32)
    default:
      set_error("small-n path supports n in {8, 16, 24, 32}");
      return TS_ERR_UNSUPPORTED;
  }
#undef TS_PROP_CASE
}

}  // namespace

bool small_n_supported(const ts_plan* p) {
  for (int k = 0; k < p->d; ++k)
    if (p->n[k] != 8 && p->n[k] != 16 && p->n[k] != 24 && p->n[k] != 32) return false;
  return true;
}

ts_status build_small_tables(ts_plan* p, cudaStream_t s) {
  for (int k = 0; k < p->d; ++k) {
    AxisTables* t = p->axis[k].get();
    std::lock_guard<std::mutex> lk(t->mu);
    if (!t->Sf32) {
      const int cnt = t->n * t->n;
      float* buf = nullptr;
      TS_TRY(table_alloc((void**)&buf, sizeof(float) * 2 * cnt, s));
      k_to_f32_table<<<(cnt + 255) / 256, 256, 0, s>>>(t->S, t->St, buf, buf + cnt, cnt);
      TS_LAUNCHED(1);
      TS_CHECK_CUDA(cudaStreamSynchronize(s));
      t->Stf32 = buf + cnt;
      t->Sf32 = buf;
      t->bytes += 8LL * cnt;
    }
    p->Sf32[k] = t->Sf32;
    p->Stf32[k] = t->Stf32;
  }
  return TS_OK;
}

// nsteps of: [theta_pre phase on the first load] -> the groups' axis propagators, one HBM
// pass per group -> [theta_post phase on the last store]; with V2 == NULL a single exact
// propagator (nsteps = 1).
ts_status small_n_propagate(const ts_plan* p, double tau, const float2* in, float2* out, const double* V2, double dt,
                            int nsteps, cudaStream_t s) {
  if (!small_n_supported(p) || !p->Sf32[0]) {
    set_error("the FP32 small-n path needs every n_k in {8, 16, 24, 32} and TS_FP32 in the plan's mask");
    return TS_ERR_UNSUPPORTED;
  }
  const std::vector<Group> gs = make_groups(p);
  const long long N = p->N;
  AxisOps ops{};
  int tot = 0;
  for (int k = 0; k < p->d; ++k) {
    ops.S[k] = p->S[k];
    ops.St[k] = p->St[k];
    ops.lam[k] = p->lam[k];
    ops.n[k] = p->n[k];
    ops.off[k] = tot;
    tot += p->n[k] * p->n[k];
  }
  void* mats = nullptr;
  void* v2f = nullptr;
  TS_TRY(scratch_alloc(&mats, sizeof(float2) * tot, s));
  ts_status st = TS_OK;
  {
    int nn = 0;
    for (int k = 0; k < p->d; ++k) nn = p->n[k] * p->n[k] > nn ? p->n[k] * p->n[k] : nn;
    k_axis_propagators<<<dim3((nn + 127) / 128, p->d), 128, 0, s>>>(ops, p->d, tau, (float2*)mats);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("axis propagator launch failed");
      st = TS_ERR_CUDA;
    }
  }
  if (st == TS_OK && V2) {
    st = scratch_alloc(&v2f, sizeof(float) * N, s);
    if (st == TS_OK) {
      k_to_f32<<<148 * 8, 256, 0, s>>>(V2, (float*)v2f, N);
      count_launches(1);
      if (cudaGetLastError() != cudaSuccess) st = TS_ERR_CUDA;
    }
  }
  const int ng = (int)gs.size();
  for (int step = 0; step < nsteps && st == TS_OK; ++step) {
    for (int gi = 0; gi < ng && st == TS_OK; ++gi) {
      const Group& g = gs[gi];
      PropParams gp{};
      const int nm = g.k1 - g.k0;
      gp.lo = 1;
      gp.hi = 1;
      for (int j = 0; j < g.k0; ++j) gp.lo *= p->n[j];
      for (int j = g.k1; j < p->d; ++j) gp.hi *= p->n[j];
      for (int j = 0; j < nm; ++j) gp.E[j] = (const float2*)mats + ops.off[g.k0 + j];
      gp.T = g.T;
      gp.V2 = (const float*)v2f;
      const bool first = gi == 0, last = gi == ng - 1;
      gp.theta_pre = (V2 && first) ? (float)(step == 0 ? 0.5 * dt : 0.0) : 0.f;
      gp.theta_post = (V2 && last) ? (float)(step == nsteps - 1 ? 0.5 * dt : dt) : 0.f;
      const float2* src = (step == 0 && first) ? in : out;
      const bool src16 = reinterpret_cast<uintptr_t>(src) % 16 == 0, out16 = reinterpret_cast<uintptr_t>(out) % 16 == 0;
      gp.pairs = gp.lo > 1 ? (gp.T % 2 == 0 && src16 && out16 ? 1 : 0) : (p->n[g.k0] % 2 == 0 && out16 ? 2 : 0);
      st = group_pass(p->n[g.k0], nm, src, out, gp, s);
    }
  }
  scratch_free(mats, s);
  scratch_free(v2f, s);
  return st;
}

}  // namespace ts
