// Fused multi-mode contraction for small axis lengths (n <= 32), complex64 data, FP32
// arithmetic: the exact propagator e^{-i tau (-Delta + V1)} (eq. exact_prop) of the 4D-9D
// problems in 2 ceil(d / f) - 1 HBM passes instead of 2d, and the Strang step (Sec. 5.1)
// with the e^{-i V2 theta} factor folded into the first and last pass.
//
// Axes are cut into groups of consecutive modes.  For a group [k0, k1) with
// lo = prod_{j<k0} n_j, G = prod_{k0<=j<k1} n_j and hi = prod_{j>=k1} n_j, a CTA owns the
// tile of T consecutive lo-indices (or, for k0 = 0, T consecutive hi-indices) times all G
// group indices: runs of >= 8 contiguous elements in HBM, so loads and stores coalesce.
// Input and output may be the same array: a CTA reads its whole tile before writing it.
// CTAs are persistent over tiles and double-buffer them: while one tile is contracted the
// next one arrives by cp.async.  In shared memory the tile is stored with every group
// extent padded to an odd length,
// so that the fibers of any mode start on distinct banks.  Each mode is contracted by
// per-thread fibers held in registers (n complex values in, n out, 2 n^2 FFMA per fiber)
// with the n x n matrix read from shared memory as broadcasts, in place.  The last group
// runs its forward modes, multiplies every coefficient by prod_k e^{-i tau lambda_k[i_k]}
// (per-axis FP32 phase tables), then its backward modes, in one pass.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "async_copy.cuh"
#include "small_n.cuh"

namespace ts {
namespace {

constexpr int SMALL_THREADS = 256;
constexpr int MAXG = 4;  // modes per group

struct GroupParams {
  int nm;                 // modes in the group
  int npad[MAXG];         // odd-padded extents in shared memory
  long long lo, hi;       // extents below / above the group
  long long G;            // product of the group's extents
  int T;                  // tile count along lo (lo > 1) or along hi (lo == 1)
  long long Gpad;         // product of padded extents
  const float* fwd[MAXG]; // forward: row-major S_k   (y_j = sum_i S_k[i][j] x_i)
  const float* bwd[MAXG]; // backward: row-major S_k^T (y_j = sum_i S_k[j][i] x_i)
  int do_fwd, do_bwd, do_phase;
  // phase of step 3 (middle pass): per-axis tables over all d axes
  int d;
  int k0;                 // first axis of the group
  int n_all[MAXD];
  const float2* ph[MAXD];
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

// Contract mode m of the tile in place along every fiber of that mode:
// y_j = sum_i M[i][j] x_i with M row-major (M = S_k: forward, M = S_k^T: backward).
// Tile-local indices are 32-bit; Tlo is a power of two (shift / mask) and N a constant.
template <int N>
__device__ void contract_mode(float2* tile, const float* M, int m, const GroupParams& p, int lgTlo, int Thi) {
  const int Tlo = 1 << lgTlo;
  int st_m = Tlo;
  for (int j = 0; j < m; ++j) st_m *= p.npad[j];
  int inner_cnt = Tlo;
  for (int j = 0; j < m; ++j) inner_cnt *= N;
  int outer_cnt = Thi;
  for (int j = m + 1; j < p.nm; ++j) outer_cnt *= N;
  const int fibers = inner_cnt * outer_cnt;
  for (int f = threadIdx.x; f < fibers; f += blockDim.x) {
    const int in_i = f % inner_cnt, out_i = f / inner_cnt;
    int addr = in_i & (Tlo - 1);
    int rem = in_i >> lgTlo, mul = Tlo;
    for (int j = 0; j < m; ++j) {
      addr += (rem % N) * mul;
      rem /= N;
      mul *= p.npad[j];
    }
    int mul2 = st_m * p.npad[m];
    int r2 = out_i;
    for (int j = m + 1; j < p.nm; ++j) {
      addr += (r2 % N) * mul2;
      r2 /= N;
      mul2 *= p.npad[j];
    }
    addr += r2 * mul2;
    float2 x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = tile[addr + i * st_m];
    // four outputs per 16-byte load of the matrix row: 8 FFMA per shared-memory load
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float4 w = *reinterpret_cast<const float4*>(M + i * N + j);
        re[0] = fmaf(w.x, x[i].x, re[0]);
        im[0] = fmaf(w.x, x[i].y, im[0]);
        re[1] = fmaf(w.y, x[i].x, re[1]);
        im[1] = fmaf(w.y, x[i].y, im[1]);
        re[2] = fmaf(w.z, x[i].x, re[2]);
        im[2] = fmaf(w.z, x[i].y, im[2]);
        re[3] = fmaf(w.w, x[i].x, re[3]);
        im[3] = fmaf(w.w, x[i].y, im[3]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) tile[addr + (j + q) * st_m] = make_float2(re[q], im[q]);
    }
  }
}

// Shared-memory index of tile element e (global order: t fastest, group indices, th) and
// its group-flattened index g (unpadded).
template <int N>
__device__ __forceinline__ int tile_index(int e, int lgTlo, const GroupParams& p, int* g_out, int* th_out) {
  const int Tlo = 1 << lgTlo;
  const int t = e & (Tlo - 1);
  int r = e >> lgTlo;
  int sidx = t, mul = Tlo, g = 0, gm = 1;
  for (int j = 0; j < p.nm; ++j) {
    const int ij = r % N;
    r /= N;
    sidx += ij * mul;
    mul *= p.npad[j];
    g += ij * gm;
    gm *= N;
  }
  *g_out = g;
  *th_out = r;
  return sidx + r * mul;
}

// First element of tile b: (l0, h0) as in the tiling described at the top.
__device__ __forceinline__ void tile_origin(long long b, int lgTlo, int Thi, const GroupParams& p, long long* l0,
                                            long long* h0) {
  if (p.lo > 1) {
    const long long lblocks = p.lo >> lgTlo;
    *l0 = (b % lblocks) << lgTlo;
    *h0 = b / lblocks;
  } else {
    *l0 = 0;
    *h0 = b * Thi;
  }
}

// Persistent over tiles with two shared-memory tile buffers: the next tile's elements are
// copied asynchronously (cp.async, one 8-byte copy per element into the padded layout)
// while the current tile is contracted, so global-load latency overlaps arithmetic.
template <int N>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_group(const float2* X, float2* Y, const GroupParams p,
                                                               long long ntiles) {
  extern __shared__ __align__(16) float2 smem[];
  const int lgT = 31 - __clz(p.T);
  const int lgTlo = p.lo > 1 ? lgT : 0;
  const int Tlo = 1 << lgTlo;
  const int Thi = p.lo > 1 ? 1 : p.T;
  const int tile_pad = Tlo * (int)p.Gpad * Thi;
  const int tile_stride = (tile_pad + 1) & ~1;  // keep every buffer 16-byte aligned
  float2* buf[2] = {smem, smem + tile_stride};
  float2* rowph = smem + 2 * tile_stride;                         // Tlo phase factors (middle pass)
  float* mats = reinterpret_cast<float*>(smem + 2 * tile_stride + ((Tlo + 1) & ~1));
  const int msz = N * N;
  for (int e = threadIdx.x; e < p.nm * msz; e += blockDim.x) {
    const int m = e / msz, q = e % msz;
    if (p.do_fwd) mats[m * msz + q] = p.fwd[m][q];
    if (p.do_bwd) mats[(p.nm + m) * msz + q] = p.bwd[m][q];
  }
  const int cnt = Tlo * (int)p.G * Thi;
  auto issue_load = [&](long long b, float2* dst) {
    long long l0, h0;
    tile_origin(b, lgTlo, Thi, p, &l0, &h0);
    const long long gbase = l0 + p.lo * p.G * h0;
    if (p.pairs == 1) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        cp_async16(dst + sidx, X + gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + p.G * th));
      }
    } else if (p.pairs == 2) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        const float2* src = X + gbase + p.lo * ((long long)g + p.G * th);
        cp_async8(dst + sidx, src);
        cp_async8(dst + sidx + 1, src + 1);
      }
    } else {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        cp_async8(dst + sidx, X + gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + p.G * th));
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
      cp_async_wait<1>();  // the current tile's group has landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float2* tile = buf[cur];
    long long l0, h0;
    tile_origin(b, lgTlo, Thi, p, &l0, &h0);
    const long long gbase = l0 + p.lo * p.G * h0;
    if (p.V2 && p.theta_pre != 0.f) {
      const int step_e = p.pairs ? 2 : 1;  // both pair kinds: (e, e + 1) at (sidx, sidx + 1)
      for (int e = step_e * threadIdx.x; e < cnt; e += step_e * blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + p.G * th);
        tile[sidx] = vphase(tile[sidx], p.theta_pre, p.V2[gidx]);
        if (p.pairs) tile[sidx + 1] = vphase(tile[sidx + 1], p.theta_pre, p.V2[gidx + 1]);
      }
      __syncthreads();
    }
    if (p.do_fwd) {
      for (int m = 0; m < p.nm; ++m) {
        contract_mode<N>(tile, mats + m * msz, m, p, lgTlo, Thi);
        __syncthreads();
      }
    }
    if (p.do_phase) {
      // phase factor of the axes below the group, one per t (the last group has no axes above)
      for (int t = threadIdx.x; t < Tlo; t += blockDim.x) {
        long long q = l0 + t;
        float2 ph = make_float2(1.f, 0.f);
        for (int k = 0; k < p.k0; ++k) {
          const int ik = (int)(q % p.n_all[k]);
          q /= p.n_all[k];
          ph = cmulf(ph, p.ph[k][ik]);
        }
        rowph[t] = ph;
      }
      __syncthreads();
      const int step_e = p.pairs == 1 ? 2 : 1;  // pairs along t share the group's phase
      for (int e = step_e * threadIdx.x; e < cnt; e += step_e * blockDim.x) {
        const int t = e & (Tlo - 1);
        int r = e >> lgTlo;
        int sidx = t, mul = Tlo;
        float2 ph = make_float2(1.f, 0.f);
        for (int j = 0; j < p.nm; ++j) {
          const int ij = r % N;
          r /= N;
          sidx += ij * mul;
          mul *= p.npad[j];
          ph = cmulf(ph, p.ph[p.k0 + j][ij]);
        }
        sidx += r * mul;
        tile[sidx] = cmulf(tile[sidx], cmulf(rowph[t], ph));
        if (p.pairs == 1) tile[sidx + 1] = cmulf(tile[sidx + 1], cmulf(rowph[t + 1], ph));
      }
      __syncthreads();
    }
    if (p.do_bwd) {
      for (int m = p.nm - 1; m >= 0; --m) {
        contract_mode<N>(tile, mats + (p.nm + m) * msz, m, p, lgTlo, Thi);
        __syncthreads();
      }
    }
    if (p.pairs) {
      for (int e = 2 * threadIdx.x; e < cnt; e += 2 * blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + p.G * th);
        float2 v0 = tile[sidx], v1 = tile[sidx + 1];
        if (p.V2 && p.theta_post != 0.f) {
          v0 = vphase(v0, p.theta_post, p.V2[gidx]);
          v1 = vphase(v1, p.theta_post, p.V2[gidx + 1]);
        }
        *reinterpret_cast<float4*>(Y + gidx) = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    } else {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int g, th;
        const int sidx = tile_index<N>(e, lgTlo, p, &g, &th);
        const long long gidx = gbase + (e & (Tlo - 1)) + p.lo * ((long long)g + p.G * th);
        float2 v = tile[sidx];
        if (p.V2 && p.theta_post != 0.f) v = vphase(v, p.theta_post, p.V2[gidx]);
        Y[gidx] = v;
      }
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
}

__global__ void k_small_phase_tables(const double* lam, double tau, float2* ph, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double s, c;
    sincos(tau * lam[i], &s, &c);
    ph[i] = make_float2((float)c, (float)-s);
  }
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

constexpr size_t TILE_BUDGET = 48 * 1024;  // bytes of one complex64 tile buffer (two per CTA)

int odd(int n) { return n | 1; }

struct Group {
  int k0, k1, T;
};

// Greedy grouping of consecutive axes whose padded tile (times T = 8, i.e. 64-byte runs)
// fits the budget; T then grows while it still fits (longer contiguous runs, fewer CTAs).
std::vector<Group> make_groups(const ts_plan* p) {
  std::vector<Group> gs;
  int k = 0;
  while (k < p->d) {
    int k1 = k + 1;
    long long gpad = odd(p->n[k]);
    while (k1 < p->d && (k1 - k) < MAXG && p->n[k1] == p->n[k] &&
           (size_t)(gpad * odd(p->n[k1]) * 8 * sizeof(float2)) <= TILE_BUDGET) {
      gpad *= odd(p->n[k1]);
      ++k1;
    }
    long long lo = 1, hi = 1;
    for (int j = 0; j < k; ++j) lo *= p->n[j];
    for (int j = k1; j < p->d; ++j) hi *= p->n[j];
    const long long along = lo > 1 ? lo : hi;
    int T = 1;
    while ((size_t)(gpad * (T * 2) * sizeof(float2)) <= TILE_BUDGET && along % (T * 2) == 0 && T < 256) T *= 2;
    gs.push_back({k, k1, T});
    k = k1;
  }
  return gs;
}

int g_small_sms = 0;

template <int N>
ts_status launch_group(const float2* X, float2* Y, const GroupParams& gp, cudaStream_t s) {
  const int Tlo = gp.lo > 1 ? gp.T : 1, Thi = gp.lo > 1 ? 1 : gp.T;
  const size_t tile_stride = ((size_t)Tlo * gp.Gpad * Thi + 1) & ~size_t(1);
  const size_t smem = sizeof(float2) * (2 * tile_stride + ((Tlo + 1) & ~1)) + sizeof(float) * 2 * gp.nm * N * N;
  static bool attr = false;
  if (!attr) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_small_group<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  if (g_small_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_small_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long tiles = gp.lo > 1 ? (gp.lo / Tlo) * gp.hi : gp.hi / Thi;
  int per_sm = 0;
  TS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_group<N>, SMALL_THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  const long long grid = tiles < (long long)g_small_sms * per_sm ? tiles : (long long)g_small_sms * per_sm;
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_small_group<N><<<(unsigned)grid, SMALL_THREADS, smem, s>>>(X, Y, gp, tiles);
  TS_LAUNCHED(1);
  if (tok) {
    const long long N_all = gp.lo * gp.G * gp.hi;
    const int modes = (gp.do_fwd ? gp.nm : 0) + (gp.do_bwd ? gp.nm : 0);
    prof_end_launch(s, tok, PROF_SMALL_PASS, 4.0 * N * (double)N_all * modes, 16.0 * (double)N_all);
  }
  return TS_OK;
}

ts_status group_pass(int n, const float2* X, float2* Y, const GroupParams& gp, cudaStream_t s) {
  switch (n) {
    case 8: return launch_group<8>(X, Y, gp, s);
    case 16: return launch_group<16>(X, Y, gp, s);
    case 24: return launch_group<24>(X, Y, gp, s);
    case 32: return launch_group<32>(X, Y, gp, s);
    default:
      set_error("small-n path supports n in {8, 16, 24, 32}");
      return TS_ERR_UNSUPPORTED;
  }
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

// nsteps of: [theta_pre phase on the first load] -> forward groups -> middle (fwd + phase
// + bwd) -> backward groups -> [theta_post phase on the last store]; with V2 == NULL a
// single exact propagator (nsteps = 1).
ts_status small_n_propagate(const ts_plan* p, double tau, const float2* in, float2* out, const double* V2, double dt,
                            int nsteps, cudaStream_t s) {
  if (!small_n_supported(p) || !p->Sf32[0]) {
    set_error("the FP32 small-n path needs every n_k in {8, 16, 24, 32} and TS_FP32 in the plan's mask");
    return TS_ERR_UNSUPPORTED;
  }
  const std::vector<Group> gs = make_groups(p);
  const long long N = p->N;
  int tot = 0, off[MAXD];
  for (int k = 0; k < p->d; ++k) {
    off[k] = tot;
    tot += p->n[k];
  }
  void* tabs = nullptr;
  void* v2f = nullptr;
  TS_TRY(scratch_alloc(&tabs, sizeof(float2) * tot, s));
  ts_status st = TS_OK;
  for (int k = 0; k < p->d && st == TS_OK; ++k) {
    k_small_phase_tables<<<(p->n[k] + 127) / 128, 128, 0, s>>>(p->lam[k], tau, (float2*)tabs + off[k], p->n[k]);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) st = TS_ERR_CUDA;
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
    for (int pass = 0; pass < 2 * ng - 1 && st == TS_OK; ++pass) {
      const bool fwd_part = pass < ng - 1;
      const bool middle = pass == ng - 1;
      const int gi = fwd_part || middle ? pass : 2 * ng - 2 - pass;
      const Group& g = gs[gi];
      GroupParams gp{};
      gp.nm = g.k1 - g.k0;
      gp.lo = 1;
      gp.hi = 1;
      gp.G = 1;
      gp.Gpad = 1;
      for (int j = 0; j < g.k0; ++j) gp.lo *= p->n[j];
      for (int j = g.k1; j < p->d; ++j) gp.hi *= p->n[j];
      for (int j = 0; j < gp.nm; ++j) {
        const int k = g.k0 + j;
        gp.npad[j] = odd(p->n[k]);
        gp.G *= p->n[k];
        gp.Gpad *= gp.npad[j];
        gp.fwd[j] = p->Sf32[k];
        gp.bwd[j] = p->Stf32[k];
      }
      gp.T = g.T;
      gp.do_fwd = fwd_part || middle;
      gp.do_bwd = !fwd_part;
      gp.do_phase = middle;
      gp.d = p->d;
      gp.k0 = g.k0;
      for (int k = 0; k < p->d; ++k) {
        gp.n_all[k] = p->n[k];
        gp.ph[k] = (const float2*)tabs + off[k];
      }
      gp.V2 = (const float*)v2f;
      const bool first = pass == 0, last = pass == 2 * ng - 2;
      gp.theta_pre = (V2 && first) ? (float)(step == 0 ? 0.5 * dt : 0.0) : 0.f;
      gp.theta_post = (V2 && last) ? (float)(step == nsteps - 1 ? 0.5 * dt : dt) : 0.f;
      const float2* src = (step == 0 && first) ? in : out;
      const bool src16 = reinterpret_cast<uintptr_t>(src) % 16 == 0, out16 = reinterpret_cast<uintptr_t>(out) % 16 == 0;
      gp.pairs = gp.lo > 1 ? (gp.T % 2 == 0 && src16 && out16 ? 1 : 0) : (p->n[g.k0] % 2 == 0 && out16 ? 2 : 0);
      st = group_pass(p->n[g.k0], src, out, gp, s);
    }
  }
  scratch_free(tabs, s);
  scratch_free(v2f, s);
  return st;
}

}  // namespace ts
