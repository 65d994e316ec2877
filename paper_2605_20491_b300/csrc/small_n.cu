// Fused multi-mode propagation for small axis lengths (n <= 32), complex64 data, in FP32
// arithmetic, and for pairs of 16- or 24-point axes in BF16X6 on the tensor cores (below):
// the exact propagator e^{-i tau (-Delta + V1)} (eq. exact_prop) of the 4D-9D problems, and
// the Strang step (Sec. 5.1) with the e^{-i V2 theta} factors folded into the passes (the
// merged factor on each step's first load, the closing half step on the last store).
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
#include "tc_ptx.cuh"

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
      // V2 through the read-only path: its loads may pass the tile stores, several in flight
#pragma unroll 4
      for (int e = step_e * threadIdx.x; e < cnt; e += step_e * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        tile[sidx] = vphase(tile[sidx], p.theta_pre, __ldg(p.V2 + gidx));
        if (p.pairs) tile[sidx + 1] = vphase(tile[sidx + 1], p.theta_pre, __ldg(p.V2 + gidx + 1));
      }
      __syncthreads();
    }
    prop_modes<N, NM, 0>(tile, mats, lgTlo, Thi);
    if (p.pairs) {
#pragma unroll 4
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        float2 v0 = tile[sidx], v1 = tile[sidx + 1];
        if (p.V2 && p.theta_post != 0.f) {
          v0 = vphase(v0, p.theta_post, __ldg(p.V2 + gidx));
          v1 = vphase(v1, p.theta_post, __ldg(p.V2 + gidx + 1));
        }
        *reinterpret_cast<float4*>(Y + gidx) = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    } else {
#pragma unroll 4
      for (int e = threadIdx.x; e < cnt; e += SMALL_THREADS) {
        int g, th;
        const int sidx = tile_offset<N, NM>(e, lgTlo, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + (long long)G * th);
        float2 v = tile[sidx];
        if (p.V2 && p.theta_post != 0.f) v = vphase(v, p.theta_post, __ldg(p.V2 + gidx));
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
// tile are cooperative (64-byte runs along t for lo > 1).
//
// Cube c occupies 512 float2 at c * 512, element (i0, i1, i2) at cube_off: the row
// i0 = 0..7 is XOR-permuted by s = (i1 >> 1) | (i2 & 1) << 2 and by c, and the low bit of
// i1 by i2 and c >> 2.  With that swizzle every warp access of the three axis passes and of
// the paired copies touches each 4-byte bank exactly twice (the 256-byte minimum of a warp
// of float2), where the padded layout i0 + 9 i1 + 81 i2 met 3-4 words per bank.  The fiber
// of a lane is then a base offset XOR a compile-time pattern of the element index.
constexpr int CUBE = 512;

__device__ __forceinline__ int cube_off(int c, int i0, int i1, int i2) {
  const int s = (i1 >> 1) | ((i2 & 1) << 2);
  return ((i0 ^ s ^ c) & 7) + 8 * ((i1 ^ (i2 & 1) ^ (c >> 2)) & 7) + 64 * i2;
}

// With vph (mode 0 only), each loaded value is first multiplied by e^{-i theta V2}, V2 of
// element i of the lane's fiber g in vph[g][i].
template <int M>
__device__ __forceinline__ void cube_mode(float2* cube, int c, const float2* Em, int lane,
                                          const float (*vph)[8] = nullptr, float theta = 0.f) {
  // fibers of mode M: 64, indexed by the two other axes (a = the lower one, b = the upper);
  // element i of a fiber sits at base ^ K(i) (+ 64 i for M = 2):
  //   M = 0: K(i) = i;  M = 1: K(i) = (i >> 1) | (i << 3);  M = 2: K(i) = 12 (i & 1)
  int base[2];
  float2 x[2][8];
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int f = lane + 32 * g, a = f & 7, b = f >> 3;
    base[g] = M == 0 ? cube_off(c, 0, a, b) : M == 1 ? cube_off(c, a, 0, b) : cube_off(c, a, b, 0);
  }
  auto off = [&](int g, int i) -> int {
    if (M == 0) return base[g] ^ i;
    if (M == 1) return base[g] ^ ((i >> 1) | (i << 3));
    return (base[g] ^ (12 * (i & 1))) + 64 * i;
  };
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[g][i] = cube[off(g, i)];
  if (M == 0 && vph) {
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[g][i] = vphase(x[g][i], theta, vph[g][i]);
  }
  float re[2][8], im[2][8];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int q = 0; q < 8; ++q) re[g][q] = im[g][q] = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const float4 e = *reinterpret_cast<const float4*>(Em + i * 8 + q);  // E[q][i], E[q+1][i]
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        re[g][q] = fmaf(e.x, x[g][i].x, re[g][q]);
        re[g][q] = fmaf(-e.y, x[g][i].y, re[g][q]);
        im[g][q] = fmaf(e.x, x[g][i].y, im[g][q]);
        im[g][q] = fmaf(e.y, x[g][i].x, im[g][q]);
        re[g][q + 1] = fmaf(e.z, x[g][i].x, re[g][q + 1]);
        re[g][q + 1] = fmaf(-e.w, x[g][i].y, re[g][q + 1]);
        im[g][q + 1] = fmaf(e.z, x[g][i].y, im[g][q + 1]);
        im[g][q + 1] = fmaf(e.w, x[g][i].x, im[g][q + 1]);
      }
    }
  }
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int q = 0; q < 8; ++q) cube[off(g, q)] = make_float2(re[g][q], im[g][q]);
}

// Tiles along lo (LO: t = cube, HBM runs of 8 along t) or along hi (th = cube, runs of 512);
// PAIRS: two adjacent elements per copy (t, t + 1 or i0, i0 + 1), 16-byte global accesses.
// The element a thread copies at step k is fixed by (tid, k), so its tile offset is a
// thread constant plus a compile-time part.
template <bool LO, bool PAIRS>
__global__ void __launch_bounds__(256, 2) k_small_cubes(const float2* X, float2* Y, const PropParams p,
                                                       long long ntiles) {
  constexpr int TSZ = 8 * CUBE;  // one tile buffer
  constexpr int EPT = PAIRS ? 2 : 1, STEPS = 4096 / (256 * EPT);
  extern __shared__ __align__(16) float2 smem[];
  float2* buf[2] = {smem, smem + TSZ};
  float2* mats = smem + 2 * TSZ;
  for (int e = threadIdx.x; e < 3 * 64; e += 256) mats[e] = p.E[e / 64][e % 64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long lo = p.lo;
  auto origin = [&](long long b) -> long long {
    if (LO) {
      const long long lblocks = lo >> 3;
      return ((b % lblocks) << 3) + lo * 512 * (b / lblocks);
    }
    return 512LL * 8 * b;
  };
  // element e = EPT tid + 256 EPT k of a tile in HBM order (LO: t fastest, then g; else g
  // fastest, then th): shared index and offset from the tile's origin
  auto sidx_of = [&](int e) -> int {
    const int c = LO ? (e & 7) : (e >> 9), g = LO ? (e >> 3) : (e & 511);
    return c * CUBE + cube_off(c, g & 7, (g >> 3) & 7, g >> 6);
  };
  auto goff_of = [&](int e) -> long long { return LO ? (long long)(e & 7) + lo * (e >> 3) : (long long)e; };
  auto issue_load = [&](long long b, float2* dst) {
    const float2* src = X + origin(b);
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
      const int e = EPT * tid + 256 * EPT * k;
      const long long go = goff_of(e);
      cp_async8(dst + sidx_of(e), src + go);
      if (PAIRS) cp_async8(dst + sidx_of(e + 1), src + go + 1);
    }
    cp_async_commit();
  };
  const bool pre = p.V2 && p.theta_pre != 0.f, post = p.V2 && p.theta_post != 0.f;
  long long b = blockIdx.x;
  if (b < ntiles) issue_load(b, buf[0]);
  int cur = 0;
  for (; b < ntiles; b += gridDim.x, cur ^= 1) {
    const long long bn = b + gridDim.x;
    const long long gbase = origin(b);
    // the tile's potential samples, loaded while the tile lands and the cubes are computed:
    // vpre[g][i] for element i of the lane's axis-0 fiber g of the warp's cube (applied as
    // the first axis loads it), vpost for the thread's stores
    float vpre[2][8], vpost[16];
    if (pre) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int f = lane + 32 * g, e0 = 8 * (f & 7) + 64 * (f >> 3);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          vpre[g][i] = p.V2[LO ? gbase + warp + lo * (e0 + i) : gbase + 512LL * warp + e0 + i];
      }
    }
    if (post) {
#pragma unroll
      for (int k = 0; k < STEPS; ++k)
#pragma unroll
        for (int q = 0; q < EPT; ++q) vpost[EPT * k + q] = p.V2[gbase + goff_of(EPT * tid + 256 * EPT * k) + q];
    }
    if (bn < ntiles) {
      issue_load(bn, buf[cur ^ 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // the tile has landed (copied by every thread)
    float2* cube = buf[cur] + warp * CUBE;
    if (pre)
      cube_mode<0>(cube, warp, mats, lane, vpre, p.theta_pre);
    else
      cube_mode<0>(cube, warp, mats, lane);
    __syncwarp();
    cube_mode<1>(cube, warp, mats + 64, lane);
    __syncwarp();
    cube_mode<2>(cube, warp, mats + 128, lane);
    __syncthreads();  // every cube is done before the cooperative store
    const float2* tile = buf[cur];
    float2* dst = Y + gbase;
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
      const int e = EPT * tid + 256 * EPT * k;
      const long long go = goff_of(e);
      float2 v0 = tile[sidx_of(e)];
      if (PAIRS) {
        float2 v1 = tile[sidx_of(e + 1)];
        if (post) {
          v0 = vphase(v0, p.theta_post, vpost[2 * k]);
          v1 = vphase(v1, p.theta_post, vpost[2 * k + 1]);
        }
        *reinterpret_cast<float4*>(dst + go) = make_float4(v0.x, v0.y, v1.x, v1.y);
      } else {
        if (post) v0 = vphase(v0, p.theta_post, vpost[k]);
        dst[go] = v0;
      }
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
}

ts_status launch_cubes(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s);

// ------------------------------------------------ tensor-core small-n pass ----
//
// The same pass for groups of two axes of length N in {16, 24} on the 5th-generation tensor
// cores (precision TS_BF16X6 on complex64 data).  Applying E_k along an axis is a real GEMM
// per fiber: with x the 2N reals (re, im interleaved) of a fiber and R_k the real 2N x 2N
// embedding of E_k (R[2j][2g] = Re E[j][g], R[2j][2g+1] = -Im E[j][g], R[2j+1][2g] =
// Im E[j][g], R[2j+1][2g+1] = Re E[j][g]), y = R_k x.  A tile is T = 16 lo (or hi) indices
// x N x N values: ROWS = 16 N fibers of the first axis, the K-major operand of one tcgen05
// GEMM (M = ROWS in blocks of 128, N = K = 2N).  Data and R_k are split into three bf16
// planes (the bf16x6 products of Henry, Tang & Heinecke).  The three planes of R_k are
// stacked along N, so each data plane is read from shared memory once per K step: plane 0
// against [R0; R1; R2] (N = 6n), plane 1 against [R0; R1] and plane 2 against R0.  The
// accumulators are X = x0 R0 (the leading product alone, which keeps the FP32 accumulation's
// truncation of the corrections off the large term), Y = x0 R1 + x1 R0 + x2 R0 and
// Z = x0 R2 + x1 R1; the epilogue forms X + (Y + Z).  The first axis's epilogue writes the
// second axis's operand (rows = fibers of the second axis) back into the same shared-memory
// planes, transposed; the second epilogue stores.  The V2 phases of a Strang step are
// applied as a step's first pass loads its tile and, for the last step's closing half
// step, as the last pass stores.  One CTA per SM, one thread per row; every wait is
// bounded.
__device__ int g_small_tc_error = 0;

template <int N>
struct SmallTc {
  static constexpr int T = 16;
  static constexpr int ROWS = T * N;            // 256 / 384
  static constexpr int MB = ROWS / 128;         // M blocks
  static constexpr int NR = 2 * N;              // reals per fiber (K and N of the GEMM)
  static constexpr int KS = NR / 16;            // 16-wide K steps
  static constexpr int PLANE_A = ROWS * 128;    // one bf16 plane, rows of 64 elements (128-byte swizzle)
  static constexpr int PLANE_B = NR / 8 * 1024;  // NR rows of R_k, 8-row atoms
  static constexpr int THREADS = ROWS;
  static constexpr int ACC = 3 * NR;            // tensor-memory columns per M block (three accumulators)
  static constexpr int SMEM = 1024 + 3 * PLANE_A + 6 * PLANE_B + 64;
  static_assert(ROWS % 128 == 0 && NR % 16 == 0 && NR <= 64, "tile shape");
  static_assert(MB * ACC <= 512, "tensor memory");
};

// Byte offset of element (row m, column k) in a K-major bf16 tile of 64-element rows with
// the 128-byte swizzle (16-byte chunk c of row m stored at chunk c ^ (m mod 8)).
__device__ __forceinline__ uint32_t sw128_off(int m, int k) {
  return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((((k >> 3) ^ m) & 7) << 4) + (k & 7) * 2);
}

// The three bf16 planes of v (each the rounding of what the previous planes leave).
__device__ __forceinline__ void split3(float v, __nv_bfloat16 (&h)[3]) {
  h[0] = __float2bfloat16_rn(v);
  float r = v - __bfloat162float(h[0]);
  h[1] = __float2bfloat16_rn(r);
  r -= __bfloat162float(h[1]);
  h[2] = __float2bfloat16_rn(r);
}

// Store the planes of the complex value (re, im) at columns (k, k + 1) of row m (k even).
// (re and im converted together: the same roundings as split3 on each.)
template <int PLANE>
__device__ __forceinline__ void store_pair3(uint8_t* planes, int m, int k, float re, float im) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(re, im);
  const float2 f0 = __bfloat1622float2(h0);
  const float r1 = re - f0.x, i1 = im - f0.y;
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(r1, i1);
  const float2 f1 = __bfloat1622float2(h1);
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(r1 - f1.x, i1 - f1.y);
  const uint32_t off = sw128_off(m, k);
  *reinterpret_cast<__nv_bfloat162*>(planes + off) = h0;
  *reinterpret_cast<__nv_bfloat162*>(planes + PLANE + off) = h1;
  *reinterpret_cast<__nv_bfloat162*>(planes + 2 * PLANE + off) = h2;
}

// One axis: the six bf16x6 products of A (rows mb*128..) and the stacked planes of R, as
// three MMAs per K step and M block: columns [0, NR) X, [NR, 2 NR) Y, [2 NR, 3 NR) Z.
template <int N>
__device__ __forceinline__ void tc_axis_mmas(const uint8_t* A, const uint8_t* B, uint32_t tmem) {
  using C = SmallTc<N>;
  constexpr uint32_t id3 = tc::idesc_bf16_f32(128, 3 * C::NR), id2 = tc::idesc_bf16_f32(128, 2 * C::NR),
                     id1 = tc::idesc_bf16_f32(128, C::NR);
  // The descriptors are rebuilt from opaque base addresses on every call: hoisted out of the
  // tile loop, 36 64-bit descriptors would stay live in every thread's registers.
  uint32_t a0, b0;
  asm volatile("mov.u32 %0, %1;" : "=r"(a0) : "r"(tc::smem_u32(A)));
  asm volatile("mov.u32 %0, %1;" : "=r"(b0) : "r"(tc::smem_u32(B)));
#pragma unroll
  for (int mb = 0; mb < C::MB; ++mb) {
    const uint32_t d = tmem + (uint32_t)(mb * C::ACC);
#pragma unroll
    for (int ks = 0; ks < C::KS; ++ks) {
      const uint64_t bd = tc::desc_sw<128>(b0 + ks * 32);
      const uint32_t a = a0 + mb * 128 * 128 + ks * 32;
      tc::mma_bf16(d, tc::desc_sw<128>(a), bd, id3, ks == 0 ? 0u : 1u);
      tc::mma_bf16(d + C::NR, tc::desc_sw<128>(a + C::PLANE_A), bd, id2, 1u);
      tc::mma_bf16(d + C::NR, tc::desc_sw<128>(a + 2 * C::PLANE_A), bd, id1, 1u);
    }
  }
}

// Row m's accumulators in its M block (columns [0, NR) X, then Y, then Z).  Lane quadrant:
// warp w reads lanes 32 (w mod 4) .. + 31.
template <int N>
__device__ __forceinline__ uint32_t tc_row_base(uint32_t tmem, int warp) {
  return tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * SmallTc<N>::ACC);
}

// Columns [c0, c0 + 16) of the row: X + (Y + Z), 8 complex values.
// (Y and Z first, then X: 32 registers of loads live at a time.)
template <int N>
__device__ __forceinline__ void tc_read16(uint32_t base, int c0, float (&v)[16]) {
  uint32_t u[16], w[16];
  tc::tmem_ld16(base + (uint32_t)(SmallTc<N>::NR + c0), u);
  tc::tmem_ld16(base + (uint32_t)(2 * SmallTc<N>::NR + c0), w);
  tc::tmem_ld_wait();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(u[i]) + __uint_as_float(w[i]);
  tc::tmem_ld16(base + (uint32_t)c0, u);
  tc::tmem_ld_wait();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(u[i]) + v[i];
}

// Byte offset, in one operand plane, of value j of this thread's run: row j T + tq (tiles
// along the lower axes, LO) or tq N + j, column 2 gq.  Rows of a run differ by T = 16 (two
// 8-row atoms) or by 1 with tq N a multiple of 8, so the offset is a thread constant plus a
// compile-time part and one XOR of the chunk index.
template <int N, bool LO>
__device__ __forceinline__ uint32_t run_off(int tq, int gq, int j) {
  constexpr int T = SmallTc<N>::T;
  if (LO) return sw128_off(tq, 2 * gq) + (uint32_t)j * (T / 8) * 1024;
  return (uint32_t)(tq * (N / 8)) * 1024 + (uint32_t)(j >> 3) * 1024 + (uint32_t)(j & 7) * 128 +
         ((((uint32_t)gq >> 2) ^ (uint32_t)j) & 7) * 16 + ((uint32_t)gq & 3) * 4;
}

template <int N, bool LO>
__global__ void __launch_bounds__(SmallTc<N>::THREADS, 1) k_small_tc(const float2* X, float2* Y,
                                                                    const PropParams p, long long ntiles) {
  using C = SmallTc<N>;
  constexpr int T = C::T, G = N * N;
  static_assert(N % 8 == 0 && T == 16, "run offsets");
  extern __shared__ uint8_t tc_raw[];
  uint8_t* A = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* B = A + 3 * C::PLANE_A;  // [axis][plane]
  uint64_t* bar = reinterpret_cast<uint64_t*>(B + 6 * C::PLANE_B);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // R_k of the group's two axes, split into planes (columns >= NR of a row are never read)
  for (int e = tid; e < 2 * C::NR * C::NR; e += C::THREADS) {
    const int ax = e / (C::NR * C::NR), n = (e / C::NR) % C::NR, k = e % C::NR;
    const float2 E = p.E[ax][(k >> 1) * N + (n >> 1)];  // ET[g][j] = E[j][g]
    const float v = (n & 1) == 0 ? ((k & 1) == 0 ? E.x : -E.y) : ((k & 1) == 0 ? E.y : E.x);
    __nv_bfloat16 h[3];
    split3(v, h);
#pragma unroll
    for (int q = 0; q < 3; ++q) *reinterpret_cast<__nv_bfloat16*>(B + (ax * 3 + q) * C::PLANE_B + sw128_off(n, k)) = h[q];
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();  // generic-proxy writes of B are read by the tensor cores
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t rbase = tc_row_base<N>(tmem, warp);
  const bool pre = p.V2 && p.theta_pre != 0.f, post = p.V2 && p.theta_post != 0.f;
  // The thread's run: fixed (t, g) = (tq, gq), the other axis's index j = 0 .. N-1.  The same
  // pair serves the load (g = g0, j = g1: value j goes to row j T + tq or tq N + j of the
  // first axis's operand), epilogue 1 (row (g1 = gq, t = tq) of the first axis's result:
  // output j0 = j goes to row j T + tq or tq N + j, column gq, of the second axis's operand)
  // and epilogue 2 (row (j0 = gq, t = tq): output (t, j0, j1 = j)).  A warp reads and
  // writes runs of consecutive t (LO) or g (tiles along the upper axes).
  const int tq = LO ? tid % T : tid / N, gq = LO ? tid / T : tid % N;
  const long long lo = p.lo;
  // element (t, g0, g1) of tile base b0 sits at b0 + t + lo (g0 + N g1) (LO) or
  // b0 + G t + g0 + N g1
  const long long run0 = LO ? tq + lo * gq : (long long)G * tq + gq;
  const long long step = LO ? lo * N : (long long)N;
  auto tile_base = [&](long long b) -> long long {
    if (!LO) return (long long)G * T * b;
    const long long lblocks = lo / T;
    return (b % lblocks) * T + lo * G * (b / lblocks);
  };
  // the tile's values in registers: all N loads of a thread in flight at once, issued for
  // the next tile while the current one is on the tensor cores
  float2 xv[N];
  float vv[N];
  auto fetch = [&](long long b) {
    const long long o = tile_base(b) + run0;
    const float2* xp = X + o;
#pragma unroll
    for (int j = 0; j < N; ++j) xv[j] = xp[step * j];
    if (pre) {
      const float* vp = p.V2 + o;
#pragma unroll
      for (int j = 0; j < N; ++j) vv[j] = vp[step * j];
    }
  };
  uint32_t phase = 0;
  long long b = blockIdx.x;
  if (b < ntiles) fetch(b);
  for (; b < ntiles; b += gridDim.x) {
    const long long o = tile_base(b) + run0;
    // 1. the tile into the first axis's operand
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float2 x = xv[j];
      if (pre) x = vphase(x, p.theta_pre, vv[j]);
      store_pair3<C::PLANE_A>(A + run_off<N, LO>(tq, gq, j), 0, 0, x.x, x.y);
    }
    tc::fence_proxy_async();
    __syncthreads();
    // 2. the first axis; the next tile's loads overlap it
    if (tid == 0) {
      tc::tc_fence_after();
      tc_axis_mmas<N>(A, B, tmem);
      tc::mma_commit(&bar[0]);
    }
    if (b + gridDim.x < ntiles) fetch(b + gridDim.x);
    tc::mbar_wait(&bar[0], phase, &g_small_tc_error, 21);
    phase ^= 1;
    tc::tc_fence_after();
    // 3. its epilogue: fiber (g1 = gq, t = tq) becomes column gq of the rows (j0, t) of the
    //    second axis's operand
#pragma unroll
    for (int c0 = 0; c0 < C::NR; c0 += 16) {
      float y[16];
      tc_read16<N>(rbase, c0, y);
#pragma unroll
      for (int i = 0; i < 16; i += 2) store_pair3<C::PLANE_A>(A + run_off<N, LO>(tq, gq, (c0 + i) >> 1), 0, 0, y[i], y[i + 1]);
    }
    tc::tc_fence_before();
    tc::fence_proxy_async();
    __syncthreads();
    // 4. the second axis
    if (tid == 0) {
      tc::tc_fence_after();
      tc_axis_mmas<N>(A, B + 3 * C::PLANE_B, tmem);
      tc::mma_commit(&bar[0]);
    }
    float vp[N];
    if (post) {
      const float* v2 = p.V2 + o;
#pragma unroll
      for (int j = 0; j < N; ++j) vp[j] = v2[step * j];
    }
    tc::mbar_wait(&bar[0], phase, &g_small_tc_error, 22);
    phase ^= 1;
    tc::tc_fence_after();
    // 5. its epilogue: row (j0 = gq, t = tq) holds the values (j1, re / im) of output
    //    (t, j0, j1), at o + step j1
    float2* yp = Y + o;
#pragma unroll
    for (int c0 = 0; c0 < C::NR; c0 += 16) {
      float y[16];
      tc_read16<N>(rbase, c0, y);
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const int j1 = (c0 + i) >> 1;
        float2 v = make_float2(y[i], y[i + 1]);
        if (post) v = vphase(v, p.theta_post, vp[j1]);
        yp[step * j1] = v;
      }
    }
    tc::tc_fence_before();
    __syncthreads();  // A and the accumulators are reused by the next tile
  }
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

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

template <bool LO, bool PAIRS>
ts_status launch_cubes_t(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (2 * 8 * CUBE + 3 * 64);
  static bool attr = false;
  if (!attr) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_cubes<LO, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  if (g_small_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_small_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long tiles = gp.lo > 1 ? (gp.lo / 8) * gp.hi : gp.hi / 8;
  int per_sm = 0;
  TS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_cubes<LO, PAIRS>, 256, smem));
  if (per_sm < 1) per_sm = 1;
  const long long grid = tiles < (long long)g_small_sms * per_sm ? tiles : (long long)g_small_sms * per_sm;
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_small_cubes<LO, PAIRS><<<(unsigned)grid, 256, smem, s>>>(X, Y, gp, tiles);
  TS_LAUNCHED(1);
  if (tok) {
    const long long N_all = gp.lo * 512LL * gp.hi;
    prof_end_launch(s, tok, PROF_SMALL_PASS, 8.0 * 8 * (double)N_all * 3, 16.0 * (double)N_all);
  }
  return TS_OK;
}

ts_status launch_cubes(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  if (gp.lo > 1) return gp.pairs ? launch_cubes_t<true, true>(X, Y, gp, s) : launch_cubes_t<true, false>(X, Y, gp, s);
  return gp.pairs ? launch_cubes_t<false, true>(X, Y, gp, s) : launch_cubes_t<false, false>(X, Y, gp, s);
}

// Whether a group can run on the tensor-core pass: two axes of length 16 or 24, tiles of
// T = 16 along lo (lo > 1) or hi (lo == 1).
bool tc_group_ok(int n, int nm, const PropParams& gp) {
  if (nm != 2 || (n != 16 && n != 24)) return false;
  return gp.lo > 1 ? gp.lo % 16 == 0 : gp.hi % 16 == 0;
}

template <int N>
ts_status launch_small_tc(const float2* X, float2* Y, const PropParams& gp, cudaStream_t s) {
  using C = SmallTc<N>;
  static bool attr = false;
  if (!attr) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_tc<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_tc<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    attr = true;
  }
  if (g_small_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_small_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long tiles = gp.lo > 1 ? (gp.lo / C::T) * gp.hi : gp.hi / C::T;
  const long long grid = tiles < g_small_sms ? tiles : g_small_sms;
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  if (gp.lo > 1)
    k_small_tc<N, true><<<(unsigned)grid, C::THREADS, C::SMEM, s>>>(X, Y, gp, tiles);
  else
    k_small_tc<N, false><<<(unsigned)grid, C::THREADS, C::SMEM, s>>>(X, Y, gp, tiles);
  TS_LAUNCHED(1);
  if (tok) {
    const long long N_all = gp.lo * (long long)N * N * gp.hi;
    // six bf16 products of a 2N x 2N real GEMM per fiber and axis, two axes
    prof_end_launch(s, tok, PROF_SMALL_PASS, 6.0 * 2.0 * 2 * (2.0 * N) * (double)N_all * 2, 16.0 * (double)N_all);
  }
  return TS_OK;
}

ts_status group_pass(int n, int nm, const float2* X, float2* Y, const PropParams& gp, cudaStream_t s,
                     bool tensor = false) {
  if (tensor && tc_group_ok(n, nm, gp)) return n == 24 ? launch_small_tc<24>(X, Y, gp, s) : launch_small_tc<16>(X, Y, gp, s);
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

ts_status small_n_error_flag(int* host_flag, bool reset, cudaStream_t s) {
  TS_CHECK_CUDA(cudaMemcpyFromSymbolAsync(host_flag, g_small_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (reset && *host_flag) {
    int zero = 0;
    TS_CHECK_CUDA(cudaMemcpyToSymbolAsync(g_small_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  }
  return TS_OK;
}

bool small_tc_applicable(const ts_plan* p) {
  if (p->d < 2) return false;
  for (int k = 0; k < p->d; ++k)
    if (p->n[k] != 8 && p->n[k] != 16 && p->n[k] != 24) return false;
  return true;
}

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

// nsteps of: [V2 phase on the first load: dt / 2 in the first step, dt later] -> the
// groups' axis propagators, one HBM pass per group; the closing dt / 2 phase on the last
// store of the last step.  With V2 == NULL a single exact propagator (nsteps = 1).
ts_status small_n_propagate(const ts_plan* p, double tau, const float2* in, float2* out, const double* V2, double dt,
                            int nsteps, cudaStream_t s, bool tensor) {
  if (!small_n_supported(p) || (!tensor && !p->Sf32[0])) {
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
      // The merged phase e^{-i V2 dt} between two steps is applied on the first pass's load
      // of the later step: the first group's tiles run along the upper axes, so its
      // potential samples are read in contiguous runs (on the last pass's store they were
      // runs of 8 to 32 bytes).  Only the last step's closing half step is applied on a store.
      gp.theta_pre = (V2 && first) ? (float)(step == 0 ? 0.5 * dt : dt) : 0.f;
      gp.theta_post = (V2 && last && step == nsteps - 1) ? (float)(0.5 * dt) : 0.f;
      const float2* src = (step == 0 && first) ? in : out;
      const bool src16 = reinterpret_cast<uintptr_t>(src) % 16 == 0, out16 = reinterpret_cast<uintptr_t>(out) % 16 == 0;
      gp.pairs = gp.lo > 1 ? (gp.T % 2 == 0 && src16 && out16 ? 1 : 0) : (p->n[g.k0] % 2 == 0 && out16 ? 2 : 0);
      st = group_pass(p->n[g.k0], nm, src, out, gp, s, tensor);
    }
  }
  scratch_free(mats, s);
  scratch_free(v2f, s);
  return st;
}

}  // namespace ts
