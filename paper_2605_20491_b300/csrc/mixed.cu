// Split-precision mode-k contraction on the 5th-generation tensor cores (tcgen05).
//
// Every contraction of the apply (steps 2 and 4 of Sec. 2.1) is the rotating-form GEMM
//     D[r][j] = sum_i X[r][i] B[j][i],   output stored transposed, Y[r + R j]
// (B[j][i] = S_k[i][j] forward, S_k[j][i] backward).  The data X and the tables B are
// carried as NP bf16 "planes" whose sum reproduces the value (x = x_0 + x_1 (+ x_2), each
// plane the bf16 rounding of what the previous planes leave), following the multi-term
// bf16 products of Henry, Tang & Heinecke (2019):
//     NP = 1 (TS_BF16X1): x0 b0                                          (~8 bits)
//     NP = 2 (TS_BF16X3): x0 b0 + x0 b1 + x1 b0                          (~16 bits)
//     NP = 3 (TS_BF16X6): x0 b0 + x0 b1 + x1 b0 + x1 b1 + x0 b2 + x2 b0  (~24 bits)
// All products of one output tile accumulate in one FP32 accumulator in tensor memory.
//
// Kernel structure: persistent (one CTA per SM, 576 threads), 128 x BN output tiles
// handed out round-robin with the N tile fastest, so that the CTAs working on the same
// 128 rows run together and share the X tile through L2:
//   warp 0 lane 0  -- TMA producer: for each K chunk (BK = 64 with the 128-byte swizzle
//                     or 32 with the 64-byte swizzle) loads the X planes (128 x BK bf16
//                     boxes) and the B planes (BN x BK) into an NS-stage ring that runs
//                     across tiles;
//   warp 1 lane 0  -- MMA issuer: tcgen05.mma kind::f16 (M = 128, N = BN, K = 16) for
//                     every (plane pair, K step) into one of two TMEM accumulator buffers;
//                     commits free the ring slots and hand the buffer to the epilogue;
//   warps 2..17    -- epilogue, overlapped with the next tile's MMAs: tcgen05.ld of the
//                     accumulator rows (warp w owns TMEM lanes 32 (w % 4) + 0..31 and
//                     every fourth 16-column chunk),
//                     optional fused pointwise step 3 (1/(Lambda + sigma) or
//                     e^{-i tau Lambda}, Lambda from per-axis tables), then either the NP
//                     bf16 planes of the next pass or the final FP64 / complex128 /
//                     complex64 result, stored transposed.
// On long real axes CTA pairs (clusters of two) share every MMA instead (cta_group::2,
// 256-row units, each CTA staging half of the B tile); see k_rot_tc.
// Complex data is planar inside the pipeline (re and im planes); a complex tile keeps
// two accumulators (re, im) that share every B tile, so the phase multiply can mix them.
#include <cudaTypedefs.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fixed.cuh"
#include "mixed.cuh"
#include "pointwise.cuh"
#include "split.cuh"
#include "tc_ptx.cuh"

namespace ts {

long long mixed_plane_elems(const ts_plan* p) {
  long long m = 0;
  for (int k = 0; k < p->d; ++k) {
    const long long e = (p->N / p->n[k]) * ((p->n[k] + 7) & ~7);
    m = e > m ? e : m;
  }
  return m;
}

int bf16_planes(ts_precision prec) {
  if (prec == TS_BF16X1) return 1;
  if (prec == TS_BF16X3) return 2;
  if (prec == TS_BF16X6) return 3;
  return 0;
}

namespace {

__device__ int g_tc_error = 0;

constexpr int BM = 128;             // rows per tile = TMEM lanes
constexpr int UMMA_K = 16;          // K of one tcgen05.mma kind::f16
constexpr int MAX_STAGES = 8;
constexpr int SMEM_LIMIT = 232448;  // 227 KB opt-in shared memory per CTA

// Scales of the fixed-point iterate U = u 2^s of a refined solve (see mixed_solve_schedule):
// fx[0] = the largest biased FP64 exponent of b (recorded by the input split), fx[1] = the
// largest biased FP32 exponent of u_0 (recorded by the pass that stores U_0).  Scale kind 0
// (U_0) follows from the bound max|u| <= beta max|b|, kind 1 (every later U) from max|u_0|;
// both keep |U| < 2^(hu - 1).
struct FixScale {
  const int* fx;
  int hu;   // headroom of the exact residual: |U| < 2^hu
  int l2b;  // ceil(log2 beta) + 2
};

__device__ __forceinline__ int fix_scale(const FixScale& f, int kind) {
  const int s0 = f.hu - (f.fx[0] - 1022) - f.l2b;
  if (kind == 0) return s0;
  int s1 = f.hu - (f.fx[1] - 126) - 1;
  s1 = s1 < s0 ? s0 : s1;
  return s1 > s0 + 60 ? s0 + 60 : s1;
}

struct EpiParams {
  int out_mode;    // 0: bf16 planes, 1: FP64 real, 2: complex128, 3: complex64, 4: FP64 real +=,
                   // 5: U = fixed(v) (int64), 6: U = U 2^ds + fixed(v), 7: FP64 (U 2^ds + fixed(v)) 2^-s
  int* emax_out;   // out_mode 1 / 4: atomic max of the stored values' biased exponents; 5: of the
                   // values' biased FP32 exponents (NULL: none)
  FixScale fxs;             // out_mode 5-7: the solve's scales
  int fix_in, fix_out;      // scale kinds of the U read (6, 7) and of the result (5-7)
  const long long* fix_src; // out_mode 6, 7: U before the update (may equal out for 6)
  int scale_mode;  // 0: none, 1: inverse 1/(Lambda + sigma), 2: phase e^{-i tau Lambda}
  long long R;     // rows of the pass
  int n;           // contracted (= output column) extent
  long long N;     // elements per plane (R * n)
  // Where output (row r, column j) goes: r_o + Ro j, planes No elements apart, with
  // r_o = (r / on) old + r % on.  Plane outputs are the next pass's input, whose fastest
  // axis (extent on) is stored in rows of old = on rounded up to a multiple of 8 (TMA rows
  // are 16-byte aligned); FP64 / complex results are unpadded (on = old = 1, Ro = R).
  long long Ro, No;
  int on, old;
  void* out;
  int nstages;
  int bn;
  double sigma;
  int rd;                     // row axes for the scale (d - 1)
  int rn[MAXD];               // their sizes, fastest first
  const double* rlam[MAXD];   // their eigenvalues (scale_mode 1)
  const double2* rph[MAXD];   // their phase tables (scale_mode 2)
  const float* clam;          // eigenvalues of the contracted axis (FP32)
  const float2* cph;          // phase table of the contracted axis (FP32)
};

template <int NP>
struct Products;
template <>
struct Products<1> {
  static constexpr int count = 1;
  __device__ static int a(int) { return 0; }
  __device__ static int b(int) { return 0; }
};
template <>
struct Products<2> {
  static constexpr int count = 3;
  __device__ static int a(int q) { return q == 2 ? 1 : 0; }
  __device__ static int b(int q) { return q == 1 ? 1 : 0; }
};
template <>
struct Products<3> {
  static constexpr int count = 6;
  // (0,0) (0,1) (1,0) (1,1) (0,2) (2,0)
  __device__ static int a(int q) { return q == 2 || q == 3 ? 1 : (q == 5 ? 2 : 0); }
  __device__ static int b(int q) { return q == 1 || q == 3 ? 1 : (q == 4 ? 2 : 0); }
};

// Epilogue warps: four per TMEM lane quarter, each draining every fourth 16-column chunk.
// The epilogue is latency-bound (TMEM load -> split -> 2-byte stores), so more warps hide
// more of it: 16 warps run the BF16X3 plane pass 8% faster than 8.
constexpr int EPI_WARPS = 16;
static_assert(EPI_WARPS % 4 == 0, "epilogue warps come in lane-quarter groups");
constexpr int TC_THREADS = 32 * (2 + EPI_WARPS);

// float -> double with integer instructions only (sign, exponent rebias +896, mantissa
// shift by 29): every FP64-pipe instruction is scarce on this GPU.  Exact for normal
// numbers; zero stays a signed zero, infinities and NaNs map to infinities and NaNs, and
// FP32 subnormals (below 1.2e-38) are flushed to zero.
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu);
  const unsigned long long e64 = e == 0u ? 0ull : (e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u));
  const unsigned long long bits =
      ((unsigned long long)(u & 0x80000000u) << 32) | (e64 << 52) | (e == 0u ? 0ull : (m << 29));
  return __longlong_as_double((long long)bits);
}

// sigma + the row axes' eigenvalues (scale 1) or the product of their phases (scale 2) at
// data row r of a pass, from the per-axis FP64 tables (the first row axis fastest).
__device__ __forceinline__ void epi_row_factors(const EpiParams& ep, long long r, float* rowsum, float2* rowph) {
  unsigned q = (unsigned)r;  // rows of a pass are below 2^31
  double sacc = ep.sigma;
  double pr = 1.0, pi = 0.0;
  for (int k = 0; k < ep.rd; ++k) {
    const unsigned qq = q / (unsigned)ep.rn[k];
    const int i = (int)(q - qq * (unsigned)ep.rn[k]);
    q = qq;
    if (ep.scale_mode == 1) {
      sacc += ep.rlam[k][i];
    } else {
      double2 ph = ep.rph[k][i];
      double tr = pr * ph.x - pi * ph.y;
      pi = pr * ph.y + pi * ph.x;
      pr = tr;
    }
  }
  *rowsum = (float)sacc;
  *rowph = make_float2((float)pr, (float)pi);
}

// Output row of data row r (see EpiParams::on).
__device__ __forceinline__ long long epi_out_row(const EpiParams& ep, long long r) {
  if (ep.on == ep.old) return r;
  const long long q = r / ep.on;
  return q * ep.old + (r - q * ep.on);
}

// The epilogue for one 16-column chunk of one accumulator row: data row r, output columns
// jbase..jbase+15 (those below ep.n), accumulator values v[component][column].  Applies the
// fused pointwise step, then stores the bf16 planes of the next pass or the final result
// (transposed: element r + R j); emx collects the largest biased exponent of FP64 stores.
template <int NP, int NACC, bool PLANES_OUT>
__device__ __forceinline__ void epi_chunk(const EpiParams& ep, const uint32_t (&v)[NACC][16], long long r, int jbase,
                                          float rowsum, float2 rowph, int& emx, int fs = 0, int fds = 0,
                                          float fsc = 0.f) {
  const int jn = ep.n - jbase < 16 ? ep.n - jbase : 16;
  long long idx = r + ep.Ro * (long long)jbase;  // r: the output row (mapped by the caller)
  // the chunk's previous values (out_mode 4: u as FP64 bits; 6, 7: the integer U), all 16
  // loads issued before any store so that they overlap
  long long prev[16];
  if (!PLANES_OUT && (ep.out_mode == 4 || (NACC == 1 && ep.out_mode >= 6))) {
    const long long* src = ep.out_mode == 4 ? reinterpret_cast<const long long*>(ep.out) : ep.fix_src;
#pragma unroll
    for (int i = 0; i < 16; ++i) prev[i] = i < jn ? src[idx + ep.Ro * (long long)i] : 0;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i, idx += ep.Ro) {
    if (i >= jn) break;
    const int j = jbase + i;
    float val[NACC];
#pragma unroll
    for (int c = 0; c < NACC; ++c) val[c] = __uint_as_float(v[c][i]);
    if (ep.scale_mode == 1) {
      // fast division (2 ulp of FP32, far below the rounding of the bf16 planes)
      val[0] = __fdividef(val[0], rowsum + ep.clam[j]);
    } else if (ep.scale_mode == 2 && NACC == 2) {
      const float2 cp = ep.cph[j];
      const float cx = cp.x, cy = cp.y;
      const float phx = rowph.x * cx - rowph.y * cy;
      const float phy = rowph.x * cy + rowph.y * cx;
      const float re = val[0] * phx - val[NACC - 1] * phy;
      const float im = val[0] * phy + val[NACC - 1] * phx;
      val[0] = re;
      val[NACC - 1] = im;
    }
    if (PLANES_OUT) {
      __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(ep.out);
#pragma unroll
      for (int c = 0; c < NACC; ++c) split_store<NP>(val[c], o + (long long)c * NP * ep.No, ep.No, idx);
    } else if (ep.out_mode == 1) {
      const double o = f2d(val[0]);
      reinterpret_cast<double*>(ep.out)[idx] = o;
      emx = max(emx, (__double2hiint(o) >> 20) & 0x7FF);
    } else if (ep.out_mode == 4) {
      const double o = __longlong_as_double(prev[i]) + f2d(val[0]);
      reinterpret_cast<double*>(ep.out)[idx] = o;
      emx = max(emx, (__double2hiint(o) >> 20) & 0x7FF);
    } else if (ep.out_mode == 2) {
      reinterpret_cast<double2*>(ep.out)[idx] = make_double2(f2d(val[0]), f2d(val[NACC - 1]));
    } else if (ep.out_mode == 3 || NACC == 2) {
      reinterpret_cast<float2*>(ep.out)[idx] = make_float2(val[0], val[NACC - 1]);
    } else if (ep.out_mode == 5) {  // the fixed-point iterate U_0 (real data only)
      // v 2^s is exact in FP32 (fsc = 2^s, nonzero when representable) and |v 2^s| < 2^62:
      // one conversion to int64, rounded to nearest
      reinterpret_cast<long long*>(ep.out)[idx] = fsc != 0.f ? __float2ll_rn(val[0] * fsc) : f32_to_fixed(val[0], fs);
      emx = max(emx, (int)((__float_as_uint(val[0]) >> 23) & 0xFFu));
    } else {  // 6, 7: U 2^ds + fixed(delta), integer addition (exact)
      const long long dq = fsc != 0.f ? __float2ll_rn(val[0] * fsc) : f32_to_fixed(val[0], fs);
      const long long un = (prev[i] << fds) + dq;
      if (ep.out_mode == 6)
        reinterpret_cast<long long*>(ep.out)[idx] = un;
      else
        reinterpret_cast<double*>(ep.out)[idx] = fixed_to_f64_rz(un, fs);
    }
  }
}

// PAIR: CTA pairs (clusters of 2) share each MMA through tcgen05 cta_group::2.  A unit is
// then 256 rows x BN columns: each CTA stages its own 128 rows of X and half (BN / 2 rows)
// of the S_k tile, the leader (rank 0) issues M = 256 MMAs that read both CTAs' shared
// memory and write both CTAs' TMEM, and each CTA's epilogue drains its own 128 rows.  Per
// SM this halves the shared-memory traffic of the S_k operand (staging and MMA reads).
// Both CTAs' TMA loads complete on the leader's stage barrier (the leader alone expects
// their bytes); commits are multicast to both CTAs; both epilogues arrive on the leader's
// accumulator-drained barrier.
template <int NP, int NACC, int BKT, bool PLANES_OUT, bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_rot_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const EpiParams ep) {
  constexpr int SW = BKT * 2;  // bytes per smem row = swizzle width
  constexpr int CL = PAIR ? 2 : 1;  // CTAs per cluster
  constexpr int CG = PAIR ? 2 : 1;   // tcgen05 CTA group
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int BN = ep.bn;
  const int NS = ep.nstages;
  const uint32_t A_TILE = BM * BKT * 2;
  const uint32_t B_TILE = (uint32_t)(PAIR ? BN / 2 : BN) * BKT * 2;
  const uint32_t A_STAGE = NACC * NP * A_TILE;
  const uint32_t B_STAGE = NP * B_TILE;
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)NS * A_STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NS * (A_STAGE + B_STAGE));
  uint64_t* full = bars;
  uint64_t* empty = bars + MAX_STAGES;
  uint64_t* accf = bars + 2 * MAX_STAGES;      // accumulator buffer b ready (MMA -> epilogue)
  uint64_t* acce = bars + 2 * MAX_STAGES + 2;  // accumulator buffer b drained (epilogue -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MAX_STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (ep.n + BKT - 1) / BKT;
  const int mtiles = (int)((ep.R + BM - 1) / BM);
  const int ntiles = (ep.n + BN - 1) / BN;
  // Work units: with CTA pairs, unit t covers M tiles (t / ntiles) * 2 + rank (one per CTA
  // of the pair) and N tile t % ntiles, and the pair splits the B tile between its two CTAs.
  // Every TMA load lands in the issuing CTA's own shared memory.
  const int rank = CL > 1 ? (int)tc::cluster_ctarank() : 0;
  const int unit0 = CL > 1 ? (int)tc::cluster_id_x() : (int)blockIdx.x;
  const int unit_step = CL > 1 ? (int)tc::cluster_count_x() : (int)gridDim.x;
  const int total = ((mtiles + CL - 1) / CL) * ntiles;
  const uint16_t cta_mask = (uint16_t)((1u << CL) - 1u);
  const uint32_t acc_cols = NACC * BN;
  uint32_t ncols = 32;
  while (ncols < 2 * acc_cols) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);  // one commit by the MMA-issuing CTA
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], PAIR ? 2 * EPI_WARPS : EPI_WARPS);  // pairs: both CTAs' epilogues
    }
    tc::fence_barrier_init();
    tc::fence_proxy_async();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 0) {
    tc::tmem_alloc<CG>(tmem_slot, ncols);
    tc::tmem_relinquish<CG>();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (CL > 1) tc::cluster_sync();  // peers' barriers are initialised before any remote use
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: a ring of NS stages that runs across tiles
      int it = 0;
      for (int t = unit0; t < total; t += unit_step) {
        const int m0 = ((t / ntiles) * CL + rank) * BM, n0 = (t % ntiles) * BN;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % NS, round = it / NS;
          if (round > 0) tc::mbar_wait(&empty[s], (round - 1) & 1, &g_tc_error, 1);
          if (PAIR) {
            // both CTAs' boxes complete on the leader's barrier; the leader expects all of them
            const uint32_t lead_full = tc::mapa_shared(&full[s], 0);
            if (rank == 0) tc::mbar_arrive_expect_tx(&full[s], 2 * (A_STAGE + B_STAGE));
            for (int c = 0; c < NACC; ++c)
              for (int p = 0; p < NP; ++p)
                tc::tma_load_3d_pair(sA + (size_t)s * A_STAGE + (c * NP + p) * A_TILE, &tmA, kc * BKT, m0,
                                     c * NP + p, lead_full);
            for (int p = 0; p < NP; ++p)
              tc::tma_load_3d_pair(sB + (size_t)s * B_STAGE + p * B_TILE, &tmB, kc * BKT, n0 + rank * (BN / 2), p,
                                   lead_full);
            continue;
          }
          tc::mbar_arrive_expect_tx(&full[s], A_STAGE + B_STAGE);
          for (int c = 0; c < NACC; ++c)
            for (int p = 0; p < NP; ++p)
              tc::tma_load_3d(sA + (size_t)s * A_STAGE + (c * NP + p) * A_TILE, &tmA, kc * BKT, m0, c * NP + p,
                              &full[s]);
          for (int p = 0; p < NP; ++p)
            tc::tma_load_3d(sB + (size_t)s * B_STAGE + p * B_TILE, &tmB, kc * BKT, n0, p, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && (!PAIR || rank == 0)) {
      // ---------------- MMA issuer (pairs: the leader only)
      const uint32_t idesc = tc::idesc_bf16_f32(PAIR ? 2 * BM : BM, BN);
      int it = 0, tl = 0;
      for (int t = unit0; t < total; t += unit_step, ++tl) {
        const int ab = tl & 1, use = tl >> 1;
        if (use > 0) tc::mbar_wait(&acce[ab], (use - 1) & 1, &g_tc_error, 4);
        tc::tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(ab * acc_cols);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int s = it % NS, round = it / NS;
          tc::mbar_wait(&full[s], round & 1, &g_tc_error, 2);
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(sA + (size_t)s * A_STAGE);
          const uint32_t b0 = tc::smem_u32(sB + (size_t)s * B_STAGE);
#pragma unroll
          for (int ks = 0; ks < BKT / UMMA_K; ++ks) {
#pragma unroll
            for (int q = 0; q < Products<NP>::count; ++q) {
              const uint64_t bdesc = tc::desc_sw<SW>(b0 + Products<NP>::b(q) * B_TILE + ks * 32);
#pragma unroll
              for (int c = 0; c < NACC; ++c) {
                const uint64_t adesc = tc::desc_sw<SW>(a0 + (c * NP + Products<NP>::a(q)) * A_TILE + ks * 32);
                if (PAIR)
                  tc::mma_bf16_pair(dbase + (uint32_t)(c * BN), adesc, bdesc, idesc, (kc | ks | q) != 0);
                else
                  tc::mma_bf16(dbase + (uint32_t)(c * BN), adesc, bdesc, idesc, (kc | ks | q) != 0);
              }
            }
          }
          if (PAIR)
            tc::mma_commit_pair(&empty[s], cta_mask);  // both CTAs' halves of the stage are free
          else
            tc::mma_commit(&empty[s]);
        }
        if (PAIR)
          tc::mma_commit_pair(&accf[ab], cta_mask);  // each CTA's TMEM holds its 128 rows
        else
          tc::mma_commit(&accf[ab]);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..EPI_WARPS+1.  Warp w reads TMEM lanes
    // 32 (w % 4) + 0..31 (tile rows) and the 16-column chunks (w - 2) / 4 + k EPI_WARPS / 4.
    const int g = warp & 3;
    const int part = (warp - 2) >> 2;  // which of the EPI_WARPS / 4 column interleaves
    int emx = 0;  // largest biased exponent stored by this thread (out_mode 1 / 4 / 5)
    int tl = 0;
    // scale of the fixed-point result and the shift of the U read (out_mode 5-7)
    const int fs = !PLANES_OUT && ep.out_mode >= 5 ? fix_scale(ep.fxs, ep.fix_out) : 0;
    const int fds = !PLANES_OUT && ep.out_mode >= 6 ? fs - fix_scale(ep.fxs, ep.fix_in) : 0;
    const float fsc = fs >= -126 && fs <= 127 ? __int_as_float((127 + fs) << 23) : 0.f;  // 2^fs
    for (int t = unit0; t < total; t += unit_step, ++tl) {
      const int ab = tl & 1, use = tl >> 1;
      const long long m0 = (long long)((t / ntiles) * CL + rank) * BM;
      const int n0 = (t % ntiles) * BN;
      tc::mbar_wait(&accf[ab], use & 1, &g_tc_error, 3);
      __syncwarp();
      tc::tc_fence_after();
      const long long r = m0 + g * 32 + lane;
      const bool row_ok = r < ep.R;
      float rowsum = 0.f;
      float2 rowph = make_float2(1.f, 0.f);
      if (ep.scale_mode != 0 && row_ok) epi_row_factors(ep, r, &rowsum, &rowph);
      const long long ro = row_ok ? epi_out_row(ep, r) : 0;
      const uint32_t lane_base = tmem + (uint32_t)(ab * acc_cols) + ((uint32_t)(g * 32) << 16);
      constexpr int CSTEP = 16 * (EPI_WARPS / 4);  // columns between a warp's chunks
      if constexpr (NACC == 1 && PLANES_OUT) {
        // real data, plane output: the next chunk's tensor-memory load is in flight while the
        // current chunk is split and stored (tcgen05.wait::ld waits for all of a thread's
        // loads, so the two register buffers alternate); the passes that write the FP64
        // result keep one buffer, as their 16 previous values already hold the registers
        uint32_t va[1][16], vb[1][16];
        int col0 = part * 16;
        if (col0 < BN) tc::tmem_ld16(lane_base + (uint32_t)col0, va[0]);
        for (; col0 < BN; col0 += 2 * CSTEP) {
          tc::tmem_ld_wait();
          const int c1 = col0 + CSTEP;
          if (c1 < BN) tc::tmem_ld16(lane_base + (uint32_t)c1, vb[0]);
          if (row_ok) epi_chunk<NP, NACC, PLANES_OUT>(ep, va, ro, n0 + col0, rowsum, rowph, emx, fs, fds, fsc);
          if (c1 >= BN) break;
          tc::tmem_ld_wait();
          const int c2 = c1 + CSTEP;
          if (c2 < BN) tc::tmem_ld16(lane_base + (uint32_t)c2, va[0]);
          if (row_ok) epi_chunk<NP, NACC, PLANES_OUT>(ep, vb, ro, n0 + c1, rowsum, rowph, emx, fs, fds, fsc);
        }
      } else {
        for (int col0 = part * 16; col0 < BN; col0 += CSTEP) {
          uint32_t v[NACC][16];
#pragma unroll
          for (int c = 0; c < NACC; ++c) tc::tmem_ld16(lane_base + (uint32_t)(c * BN + col0), v[c]);
          tc::tmem_ld_wait();
          if (!row_ok) continue;
          epi_chunk<NP, NACC, PLANES_OUT>(ep, v, ro, n0 + col0, rowsum, rowph, emx, fs, fds, fsc);
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR)
          tc::mbar_arrive_cluster_relaxed(tc::mapa_shared(&acce[ab], 0));  // the leader reuses the buffer
        else
          tc::mbar_arrive_relaxed(&acce[ab]);
      }
    }
    if (!PLANES_OUT && ep.emax_out) {
      for (int o = 16; o > 0; o >>= 1) emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
      if (lane == 0) atomicMax(ep.emax_out, emx);
    }
  }
  __syncwarp();
  tc::tc_fence_before();
  __syncthreads();
  if (CL > 1) tc::cluster_sync();  // no CTA leaves while a peer may still write into it
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc<CG>(tmem, ncols);
  }
}

// ------------------------------------------------------- work-list pass ----
//
// One launch over a work list of (request, pass) items, e.g. pass s of every request of a
// serving batch: the tiles of all items form one unit space (item by item, N tile fastest
// within an item) that persistent single CTAs walk exactly like k_rot_tc walks one pass.
// Items share the template parameters (planes, components, output kind) but each has its
// own tensor maps, contracted extent n, rows R, N tile and epilogue (all in the kernel's
// parameter space); shared memory and TMEM are sized for the widest N tile of the list.
constexpr int TC_LIST_MAX = 40;
struct TcItem {
  CUtensorMap tmA;       // data planes [NACC * NP][R][n], 128-row boxes
  CUtensorMap tmB;       // S_k planes [NP][n][n], ep.bn-row boxes
  EpiParams ep;          // ep.bn: this item's N tile
  long long unit_begin;  // first unit of the item in the launch's unit space
  int mtiles, ntiles, nk;
};
struct TcItemList {
  TcItem item[TC_LIST_MAX];
  int count;
  long long total;  // units of all items
  int bn_max;       // rows of the B tile slots in shared memory
  int nstages;
};
static_assert(sizeof(TcItemList) < 32000, "the work list travels in the kernel's parameter space");

template <int NP, int NACC, int BKT, bool PLANES_OUT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_rot_tc_list(const __grid_constant__ TcItemList L) {
  constexpr int SW = BKT * 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int BNM = L.bn_max;
  const int NS = L.nstages;
  const uint32_t A_TILE = BM * BKT * 2;
  const uint32_t B_TILE = (uint32_t)BNM * BKT * 2;  // slot size; an item fills ep.bn rows of it
  const uint32_t A_STAGE = NACC * NP * A_TILE;
  const uint32_t B_STAGE = NP * B_TILE;
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)NS * A_STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NS * (A_STAGE + B_STAGE));
  uint64_t* full = bars;
  uint64_t* empty = bars + MAX_STAGES;
  uint64_t* accf = bars + 2 * MAX_STAGES;
  uint64_t* acce = bars + 2 * MAX_STAGES + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MAX_STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t acc_cols = NACC * BNM;
  uint32_t ncols = 32;
  while (ncols < 2 * acc_cols) ncols <<= 1;
  // item of unit t: the items' unit ranges are consecutive, and each role visits units in
  // increasing order, so a cursor that only moves forward finds it
  auto advance = [&](int& cur, long long t) {
    while (cur + 1 < L.count && t >= L.item[cur + 1].unit_begin) ++cur;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], EPI_WARPS);
    }
    tc::fence_barrier_init();
    tc::fence_proxy_async();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int it = 0, cur = 0;
      for (long long t = blockIdx.x; t < L.total; t += gridDim.x) {
        advance(cur, t);
        const TcItem& I = L.item[cur];
        const long long u = t - I.unit_begin;
        const int m0 = (int)(u / I.ntiles) * BM, n0 = (int)(u % I.ntiles) * I.ep.bn;
        const uint32_t bytes = A_STAGE + (uint32_t)NP * I.ep.bn * BKT * 2;
        for (int kc = 0; kc < I.nk; ++kc, ++it) {
          const int s = it % NS, round = it / NS;
          if (round > 0) tc::mbar_wait(&empty[s], (round - 1) & 1, &g_tc_error, 1);
          tc::mbar_arrive_expect_tx(&full[s], bytes);
          for (int c = 0; c < NACC; ++c)
            for (int p = 0; p < NP; ++p)
              tc::tma_load_3d(sA + (size_t)s * A_STAGE + (c * NP + p) * A_TILE, &I.tmA, kc * BKT, m0, c * NP + p,
                              &full[s]);
          for (int p = 0; p < NP; ++p)
            tc::tma_load_3d(sB + (size_t)s * B_STAGE + p * B_TILE, &I.tmB, kc * BKT, n0, p, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, tl = 0, cur = 0;
      for (long long t = blockIdx.x; t < L.total; t += gridDim.x, ++tl) {
        advance(cur, t);
        const TcItem& I = L.item[cur];
        const int BN = I.ep.bn;
        const uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        const int ab = tl & 1, use = tl >> 1;
        if (use > 0) tc::mbar_wait(&acce[ab], (use - 1) & 1, &g_tc_error, 4);
        tc::tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(ab * acc_cols);
        for (int kc = 0; kc < I.nk; ++kc, ++it) {
          const int s = it % NS, round = it / NS;
          tc::mbar_wait(&full[s], round & 1, &g_tc_error, 2);
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(sA + (size_t)s * A_STAGE);
          const uint32_t b0 = tc::smem_u32(sB + (size_t)s * B_STAGE);
#pragma unroll
          for (int ks = 0; ks < BKT / UMMA_K; ++ks) {
#pragma unroll
            for (int q = 0; q < Products<NP>::count; ++q) {
              const uint64_t bdesc = tc::desc_sw<SW>(b0 + Products<NP>::b(q) * B_TILE + ks * 32);
#pragma unroll
              for (int c = 0; c < NACC; ++c) {
                const uint64_t adesc = tc::desc_sw<SW>(a0 + (c * NP + Products<NP>::a(q)) * A_TILE + ks * 32);
                tc::mma_bf16(dbase + (uint32_t)(c * BN), adesc, bdesc, idesc, (kc | ks | q) != 0);
              }
            }
          }
          tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(&accf[ab]);
      }
    }
  } else {
    // ---------------- epilogue (as in k_rot_tc, per item)
    const int g = warp & 3;
    const int part = (warp - 2) >> 2;
    int emx = 0, tl = 0, cur = 0;
    for (long long t = blockIdx.x; t < L.total; t += gridDim.x, ++tl) {
      advance(cur, t);
      const TcItem& I = L.item[cur];
      const EpiParams& ep = I.ep;
      const int BN = ep.bn;
      const long long u = t - I.unit_begin;
      const long long m0 = (u / I.ntiles) * BM;
      const int n0 = (int)(u % I.ntiles) * BN;
      const int ab = tl & 1, use = tl >> 1;
      tc::mbar_wait(&accf[ab], use & 1, &g_tc_error, 3);
      __syncwarp();
      tc::tc_fence_after();
      const long long r = m0 + g * 32 + lane;
      const bool row_ok = r < ep.R;
      float rowsum = 0.f;
      float2 rowph = make_float2(1.f, 0.f);
      if (ep.scale_mode != 0 && row_ok) epi_row_factors(ep, r, &rowsum, &rowph);
      const long long ro = row_ok ? epi_out_row(ep, r) : 0;
      const uint32_t lane_base = tmem + (uint32_t)(ab * acc_cols) + ((uint32_t)(g * 32) << 16);
      for (int col0 = part * 16; col0 < BN; col0 += 16 * (EPI_WARPS / 4)) {
        uint32_t v[NACC][16];
#pragma unroll
        for (int c = 0; c < NACC; ++c) tc::tmem_ld16(lane_base + (uint32_t)(c * BN + col0), v[c]);
        tc::tmem_ld_wait();
        if (!row_ok) continue;
        epi_chunk<NP, NACC, PLANES_OUT>(ep, v, ro, n0 + col0, rowsum, rowph, emx);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive_relaxed(&acce[ab]);
    }
    (void)emx;  // the exponent collection of the refined solve is not used by list passes
  }
  __syncwarp();
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// ------------------------------------------------------------ pointwise ----

// FP64 / complex input -> planar bf16 planes [c][p][rows][ld0] (rows of axis 1, padded to
// ld0 = n0 rounded up to a multiple of 8); x rounded to FP32 first (the planes carry at most
// 24 bits), then split exactly in FP32.
// PADDED = false: rows need no padding (n0 % 8 == 0), element i goes to i.
// emax (MODE 0, may be NULL): raised to the largest biased FP64 exponent of the input.
template <int NP, int MODE, bool PADDED>  // MODE 0: real FP64, 1: complex128, 2: complex64
__global__ void k_split_input(const void* in, __nv_bfloat16* planes, long long N, int n0, int* emax = nullptr) {
  const int NC = MODE == 0 ? 1 : 2;
  const int ld0 = PADDED ? (n0 + 7) & ~7 : n0;  // padded row (axis 1) of the planes
  const long long Np = PADDED ? (N / n0) * ld0 : N;  // plane stride
  int emx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    long long ip = i;
    if (PADDED) {
      const long long row = i / n0;
      ip = row * ld0 + (i - row * n0);
    }
    float v[2];
    if (MODE == 0) {
      const double x = reinterpret_cast<const double*>(in)[i];
      emx = max(emx, (__double2hiint(x) >> 20) & 0x7FF);
      v[0] = (float)x;
    } else if (MODE == 1) {
      double2 z = reinterpret_cast<const double2*>(in)[i];
      v[0] = (float)z.x;
      v[1] = (float)z.y;
    } else {
      float2 z = reinterpret_cast<const float2*>(in)[i];
      v[0] = z.x;
      v[1] = z.y;
    }
    for (int c = 0; c < NC; ++c) split_store<NP>(v[c], planes + (long long)c * NP * Np, Np, ip);
  }
  if (MODE == 0 && emax) {
    for (int o = 16; o > 0; o >>= 1) emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(emax, emx);
  }
}

// The same for real FP64 input on unpadded rows, four values per thread and step (two
// 16-byte loads, one 8-byte store per plane), so that enough bytes are in flight to cover
// HBM latency; in 16-byte aligned, planes 8-byte aligned, N a multiple of 4.
template <int NP>
__global__ void k_split_real4(const double* __restrict__ in, __nv_bfloat16* __restrict__ planes, long long N,
                              int* emax) {
  const long long n4 = N >> 2;
  int emx = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    const double2 a = reinterpret_cast<const double2*>(in)[2 * q];
    const double2 b = reinterpret_cast<const double2*>(in)[2 * q + 1];
    if (emax)
      emx = max(max(max(emx, (__double2hiint(a.x) >> 20) & 0x7FF), max((__double2hiint(a.y) >> 20) & 0x7FF,
                                                                       (__double2hiint(b.x) >> 20) & 0x7FF)),
                (__double2hiint(b.y) >> 20) & 0x7FF);
    float r[4] = {(float)a.x, (float)a.y, (float)b.x, (float)b.y};
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      __nv_bfloat16 h[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        h[c] = __float2bfloat16_rn(r[c]);
        r[c] -= __bfloat162float(h[c]);
      }
      uint2 w;
      w.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
      w.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
      reinterpret_cast<uint2*>(planes + (long long)p * N)[q] = w;
    }
  }
  if (emax) {
    for (int o = 16; o > 0; o >>= 1) emx = max(emx, __shfl_xor_sync(0xffffffffu, emx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(emax, emx);
  }
}

// The input split of many items in one launch: item q owns blocks [block_begin_q,
// block_begin_{q+1}) and runs k_split_input's loop over its N values with them.
struct SplitItem {
  const void* in;
  __nv_bfloat16* planes;
  long long N;
  int n0;    // extent of axis 1 (plane rows are padded to a multiple of 8)
  int mode;  // 0: real FP64, 1: complex128, 2: complex64
  int block_begin;
};
struct SplitList {
  SplitItem item[TC_LIST_MAX];
  int count;
};

template <int NP>
__global__ void k_split_list(const __grid_constant__ SplitList L) {
  int cur = 0;
  while (cur + 1 < L.count && (int)blockIdx.x >= L.item[cur + 1].block_begin) ++cur;
  const SplitItem& I = L.item[cur];
  const int nb = (cur + 1 < L.count ? L.item[cur + 1].block_begin : (int)gridDim.x) - I.block_begin;
  const int nc = I.mode == 0 ? 1 : 2;
  const int ld0 = (I.n0 + 7) & ~7;
  const long long Np = (I.N / I.n0) * ld0;
  for (long long i = (long long)(blockIdx.x - I.block_begin) * blockDim.x + threadIdx.x; i < I.N;
       i += (long long)nb * blockDim.x) {
    long long ip = i;
    if (ld0 != I.n0) {
      const long long row = i / I.n0;
      ip = row * ld0 + (i - row * I.n0);
    }
    float v[2];
    if (I.mode == 0) {
      v[0] = (float)reinterpret_cast<const double*>(I.in)[i];
      v[1] = 0.f;
    } else if (I.mode == 1) {
      const double2 z = reinterpret_cast<const double2*>(I.in)[i];
      v[0] = (float)z.x;
      v[1] = (float)z.y;
    } else {
      const float2 z = reinterpret_cast<const float2*>(I.in)[i];
      v[0] = z.x;
      v[1] = z.y;
    }
    for (int c = 0; c < nc; ++c) split_store<NP>(v[c], I.planes + (long long)c * NP * Np, Np, ip);
  }
}

// FP64 table -> NP bf16 planes (FP64 arithmetic; tables are tiny).
// dst[p][j][i] = plane p of the split of src[i][j] (n x n): the transpose, so that the
// contracted index of the operand is contiguous (K-major); rows of ld = n rounded up to a
// multiple of 8 (16-byte TMA rows), planes n * ld apart.  The padding is left as it is
// (the caller zeroes it; TMA never reads past column n of the declared extent anyway).
__global__ void k_split_table_t(const double* src, __nv_bfloat16* dst, int n, int np) {
  const long long count = (long long)n * n;
  const int ld = (n + 7) & ~7;
  const long long pstride = (long long)n * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    double x = src[e];
    for (int p = 0; p < np; ++p) {
      __nv_bfloat16 h = __double2bfloat16(x);
      dst[p * pstride + j * ld + i] = h;
      x -= (double)__bfloat162float(h);
    }
  }
}

// ph[i] = e^{-i tau lambda_i} = (cos(tau lambda_i), -sin(tau lambda_i)) in FP64, and the
// same rounded to FP32 in phf (the per-element column factor of the epilogue).
__global__ void k_phase_table(const double* lam, double tau, double2* ph, float2* phf, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double s, c;
    sincos(tau * lam[i], &s, &c);
    ph[i] = make_double2(c, -s);
    phf[i] = make_float2((float)c, (float)-s);
  }
}

// ----------------------------------------- residual of the fixed-point iterate ----
//
// r = b - (-Delta_h + V1 + sigma) u for the iterate held as U = u 2^s (int64), d = 3, one
// spacing h: the integer R = 6 U - (six neighbours) + ((Q_xy + Q_z) U >> F), with Q the
// fixed-point tables of (sigma + V1) h^2 (F fraction bits), is exact; r = b - h^-2 2^-s R (one
// int64 -> FP64 conversion and one FMA), split into NP bf16 planes.  A CTA marches a
// 32 x 16 tile of axes (0, 1) along axis 2.  Every plane's U tile (with its one-cell halo)
// and b tile arrive by TMA into a ring of shared-memory stages; the zero fill of boxes
// reaching past the grid supplies the Dirichlet zeros, so the threads do no load address
// arithmetic and no conversion of U.
constexpr int FX_MX = 32, FX_MY = 16, FX_MZ = 64, FX_RD = 4;
constexpr int FX_UW = FX_MX + 4;  // U tile row: x0 - 2 .. x0 + 33 (a TMA box starts at an even x)
constexpr int FX_UH = FX_MY + 2;  // rows y0 - 1 .. y0 + 16
constexpr int FX_U_BYTES = FX_UW * FX_UH * 8;
constexpr int FX_B_BYTES = FX_MX * FX_MY * 8;
// a tensor TMA writes shared memory at 128-byte aligned addresses: both tiles of a stage
// start on one (the stages themselves are 128-byte multiples from a 128-byte aligned base)
constexpr int FX_B_OFF = (FX_U_BYTES + 127) / 128 * 128;
constexpr int FX_STAGE = (FX_B_OFF + FX_B_BYTES + 127) / 128 * 128;
static_assert(FX_B_OFF % 128 == 0 && FX_STAGE % 128 == 0, "TMA destinations must be 128-byte aligned");
constexpr int FX_SMEM = 128 + FX_RD * FX_STAGE + 8 * FX_RD;

struct FixResidual {
  int n0, n1, n2;
  int F;               // fraction bits of the Q tables
  const long long* Q;  // Q[0] = sigma h^2, then f_0 h^2 (n0), f_1 h^2 (n1), f_2 h^2 (n2)
  double ih2;          // h^-2
  FixScale fxs;
  int s_kind;          // scale kind of U
  const long long* U;  // the iterate (for the plane below a CTA's first plane)
  __nv_bfloat16* planes;
  long long Np;        // elements per plane
  int ld0;             // axis-0 rows of the planes, padded to a multiple of 8
};

template <int NP>
__global__ void __launch_bounds__(256) k_residual_fixu(const __grid_constant__ CUtensorMap tmU,
                                                       const __grid_constant__ CUtensorMap tmB,
                                                       const FixResidual prm) {
  extern __shared__ uint8_t fx_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(fx_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + FX_RD * FX_STAGE);
  const int n0 = prm.n0, n1 = prm.n1, n2 = prm.n2;
  const int tiles0 = (n0 + FX_MX - 1) / FX_MX, tiles1 = (n1 + FX_MY - 1) / FX_MY;
  int bid = blockIdx.x;
  const int t0 = bid % tiles0;
  bid /= tiles0;
  const int t1 = bid % tiles1;
  const int z0 = (bid / tiles1) * FX_MZ, z1 = min(z0 + FX_MZ, n2);
  const int x0 = t0 * FX_MX, y0 = t1 * FX_MY;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int x = x0 + lx, ya = y0 + ly, yb = ya + 8;
  const bool va = x < n0 && ya < n1, vb = x < n0 && yb < n1;
  const int sc = fix_scale(prm.fxs, prm.s_kind);
  const double cs = ldexp(prm.ih2, -sc);
  const long long qa = va ? prm.Q[0] + prm.Q[1 + x] + prm.Q[1 + n0 + ya] : 0;
  const long long qb = vb ? prm.Q[0] + prm.Q[1 + x] + prm.Q[1 + n0 + yb] : 0;
  const long long* q2 = prm.Q + 1 + n0 + n1;
  const int nplanes = z1 - z0 + 1;  // planes z0 .. z1 (z1 == n2 reads the zero fill)
  if (threadIdx.x == 0) {
    for (int k = 0; k < FX_RD; ++k) tc::mbar_init(&full[k], 1);
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmU);
    tc::prefetch_tmap(&tmB);
  }
  __syncthreads();
  auto issue = [&](int j) {  // plane z0 + j into stage j % FX_RD
    uint8_t* st = base + (j % FX_RD) * FX_STAGE;
    uint64_t* bar = &full[j % FX_RD];
    tc::mbar_arrive_expect_tx(bar, FX_U_BYTES + FX_B_BYTES);
    tc::tma_load_3d(st, &tmU, x0 - 2, y0 - 1, z0 + j, bar);
    tc::tma_load_3d(st + FX_B_OFF, &tmB, x0, y0, z0 + j, bar);
  };
  if (threadIdx.x == 0)
    for (int j = 0; j < FX_RD && j < nplanes; ++j) issue(j);
  const long long s2 = (long long)n0 * n1;
  long long Uda = va && z0 > 0 ? prm.U[(long long)(z0 - 1) * s2 + (long long)ya * n0 + x] : 0;
  long long Udb = vb && z0 > 0 ? prm.U[(long long)(z0 - 1) * s2 + (long long)yb * n0 + x] : 0;
  const long long ps2 = (long long)prm.ld0 * n1;
  __nv_bfloat16* pa = prm.planes + (long long)z0 * ps2 + (long long)ya * prm.ld0 + x;
  __nv_bfloat16* pb = pa + 8LL * prm.ld0;
  const int ca = (ly + 1) * FX_UW + lx + 2, cb = ca + 8 * FX_UW;  // own cells in the U tile
  for (int z = z0; z < z1; ++z) {
    const int j = z - z0;
    tc::mbar_wait(&full[j % FX_RD], (j / FX_RD) & 1, &g_tc_error, 11);
    tc::mbar_wait(&full[(j + 1) % FX_RD], ((j + 1) / FX_RD) & 1, &g_tc_error, 11);
    const long long* Uc = reinterpret_cast<const long long*>(base + (j % FX_RD) * FX_STAGE);
    const long long* Uu = reinterpret_cast<const long long*>(base + ((j + 1) % FX_RD) * FX_STAGE);
    const double* Bc = reinterpret_cast<const double*>(base + (j % FX_RD) * FX_STAGE + FX_B_OFF);
    const long long ua = Uc[ca], ub = Uc[cb];
    const long long qz = q2[z];
    const long long Ra = 6 * ua - Uc[ca - 1] - Uc[ca + 1] - Uc[ca - FX_UW] - Uc[ca + FX_UW] - Uda - Uu[ca] +
                         mul_shift(qa + qz, ua, prm.F);
    const long long Rb = 6 * ub - Uc[cb - 1] - Uc[cb + 1] - Uc[cb - FX_UW] - Uc[cb + FX_UW] - Udb - Uu[cb] +
                         mul_shift(qb + qz, ub, prm.F);
    if (va) split_store<NP>(f64_to_f32(fma(-cs, __ll2double_rn(Ra), Bc[ly * FX_MX + lx])), pa, prm.Np, 0);
    if (vb) split_store<NP>(f64_to_f32(fma(-cs, __ll2double_rn(Rb), Bc[(ly + 8) * FX_MX + lx])), pb, prm.Np, 0);
    pa += ps2;
    pb += ps2;
    Uda = ua;
    Udb = ub;
    __syncthreads();  // every thread is done with plane z: its stage takes plane z + FX_RD
    if (threadIdx.x == 0 && j + FX_RD < nplanes) issue(j + FX_RD);
  }
}

// ------------------------------------------------------------ host side ----

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3D bf16 tensor map over planes [planes][rows][cols] (cols contiguous, rows of
// ld = cols rounded up to a multiple of 8, planes ld * rows apart), box
// {box_cols cols, box_rows rows, 1 plane}, swizzle = 2 * box_cols bytes (128 or 64),
// zero fill out of bounds (so a row's padding and the K tail read as zeros).
ts_status make_map(CUtensorMap* m, const void* base, long long cols, long long rows, int planes, int box_cols,
                   int box_rows) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return TS_ERR_CUDA;
  }
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  const long long ld = (cols + 7) & ~7LL;
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(ld * rows * 2)};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for cols=%lld rows=%lld planes=%d", (int)r, cols, rows, planes);
    return TS_ERR_CUDA;
  }
  return TS_OK;
}

// 3D tensor map over an n0 x n1 x n2 array of 8-byte elements (n0 fastest, unpadded,
// n0 * 8 a multiple of 16), box {b0, b1, 1}, no swizzle, zero fill out of bounds.
ts_status make_map_8b(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int n0, int n1, int n2, int b0,
                      int b1) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return TS_ERR_CUDA;
  }
  cuuint64_t dims[3] = {(cuuint64_t)n0, (cuuint64_t)n1, (cuuint64_t)n2};
  cuuint64_t strides[2] = {(cuuint64_t)n0 * 8, (cuuint64_t)n0 * n1 * 8};
  cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d x %d array", (int)r, n0, n1, n2);
    return TS_ERR_CUDA;
  }
  return TS_OK;
}

int g_num_sms = 0;

// The residual of the fixed-point iterate into np bf16 planes (see k_residual_fixu).
ts_status residual_fixu(const ts_plan* p, const long long* U, const double* b, const long long* Q, int F,
                        const FixScale& fxs, int s_kind, __nv_bfloat16* planes, int np, cudaStream_t s) {
  CUtensorMap mu, mb;
  TS_TRY(make_map_8b(&mu, U, CU_TENSOR_MAP_DATA_TYPE_INT64, p->n[0], p->n[1], p->n[2], FX_UW, FX_UH));
  TS_TRY(make_map_8b(&mb, b, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, p->n[0], p->n[1], p->n[2], FX_MX, FX_MY));
  FixResidual prm{};
  prm.n0 = p->n[0];
  prm.n1 = p->n[1];
  prm.n2 = p->n[2];
  prm.F = F;
  prm.Q = Q;
  const double h = 2.0 * p->L[0] / (p->n[0] + 1);
  prm.ih2 = 1.0 / (h * h);
  prm.fxs = fxs;
  prm.s_kind = s_kind;
  prm.U = U;
  prm.planes = planes;
  prm.ld0 = (p->n[0] + 7) & ~7;
  prm.Np = (long long)prm.ld0 * p->n[1] * p->n[2];
  static bool attr_set[4] = {};
  const long long blocks = (long long)((p->n[0] + FX_MX - 1) / FX_MX) * ((p->n[1] + FX_MY - 1) / FX_MY) *
                           ((p->n[2] + FX_MZ - 1) / FX_MZ);
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
#define TS_FIXU(NP)                                                                                       \
  if (np == NP) {                                                                                         \
    if (!attr_set[NP]) {                                                                                  \
      TS_CHECK_CUDA(cudaFuncSetAttribute(k_residual_fixu<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         FX_SMEM));                                                       \
      attr_set[NP] = true;                                                                                \
    }                                                                                                     \
    k_residual_fixu<NP><<<(unsigned)blocks, 256, FX_SMEM, s>>>(mu, mb, prm);                              \
  }
  TS_FIXU(1) else TS_FIXU(2) else TS_FIXU(3)
#undef TS_FIXU
  TS_LAUNCHED(1);
  if (tok) prof_end_launch(s, tok, PROF_RESIDUAL, 0.0, (16.0 + 2.0 * np) * (double)p->N);
  return TS_OK;
}

template <int NP, int NACC, int BKT, bool PO, bool PAIR>
ts_status launch_pass_t(const __nv_bfloat16* A, const __nv_bfloat16* B, long long R, int n, EpiParams ep,
                        int bn_cap, cudaStream_t s) {
  constexpr int CL = PAIR ? 2 : 1;
  // pairs: N tiles in multiples of 32 (every such N is a valid M = 256 shape)
  const int bq = PAIR ? 32 : 16;
  int bn = ((n + bq - 1) / bq) * bq;
  if (bn > bn_cap) bn = bn_cap;
  if (PAIR && bn % 32 != 0) {
    set_error("CTA pairs need an N-tile cap that is a multiple of 32 (got %d)", bn_cap);
    return TS_ERR_UNSUPPORTED;
  }
  const int b_rows = PAIR ? bn / 2 : bn;  // rows of the S_k tile staged per CTA (bn % 16 == 0)
  const int stage = NACC * NP * BM * BKT * 2 + NP * b_rows * BKT * 2;
  const int reserve = 1024 + 8 * (2 * MAX_STAGES + 6);
  int ns = (SMEM_LIMIT - reserve) / stage;
  if (ns > MAX_STAGES) ns = MAX_STAGES;
  if (ns < 2) {
    set_error("tile does not fit in shared memory");
    return TS_ERR_UNSUPPORTED;
  }
  const int smem = ns * stage + reserve;
  CUtensorMap ma, mb;
  TS_TRY(make_map(&ma, A, n, R, NACC * NP, BKT, BM));
  TS_TRY(make_map(&mb, B, n, n, NP, BKT, PAIR ? bn / 2 : bn));
  ep.R = R;
  ep.n = n;
  ep.N = R * n;
  if (ep.Ro == 0) {  // unpadded output (callers set the layout of plane outputs)
    ep.Ro = R;
    ep.No = R * n;
    ep.on = ep.old = 1;
  }
  ep.bn = bn;
  ep.nstages = ns;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    TS_CHECK_CUDA(
        cudaFuncSetAttribute(k_rot_tc<NP, NACC, BKT, PO, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_LIMIT));
    attr_set = true;
  }
  if (g_num_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const long long mtiles = (R + BM - 1) / BM, ntiles = (n + bn - 1) / bn;
  const long long units = ((mtiles + CL - 1) / CL) * ntiles;
  TS_REQUIRE(units * CL < (1LL << 31), "too many tiles");
  const long long max_clusters = g_num_sms / CL;
  const unsigned grid = (unsigned)((units < max_clusters ? units : max_clusters) * CL);
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  if (CL == 1) {
    k_rot_tc<NP, NACC, BKT, PO, false><<<grid, TC_THREADS, smem, s>>>(ma, mb, ep);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TS_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_rot_tc<NP, NACC, BKT, PO, PAIR>, ma, mb, ep));
  }
  TS_LAUNCHED(1);
  if (tok) {
    const double flops = 2.0 * Products<NP>::count * NACC * (double)R * n * n;
    const double bytes = (double)NACC * R * n * 2.0 * NP * (ep.out_mode == 0 ? 2.0 : 1.0) +
                         (ep.out_mode == 1 || ep.out_mode == 3 || ep.out_mode == 5 ? 8.0
                          : ep.out_mode == 0 ? 0.0 : 16.0) * R * n;
    const int kind = ep.out_mode != 0 ? PROF_TC_PASS_OUT : (NP == 1 ? PROF_TC_PASS_X1 : PROF_TC_PASS);
    prof_end_launch(s, tok, kind, flops, bytes);
  }
  return TS_OK;
}

// Tile configuration of one pass (the autotuner's search space): K chunk 64 (128-byte
// swizzle) or 32 (64-byte swizzle), and the cap on the N tile.
struct TcConfig {
  int bk = 64;
  int bn_cap = 256;
  bool pair = false;  // CTA pairs sharing each MMA (cta_group::2, 256-row units)
};

std::mutex g_cfg_mu;
std::map<std::pair<int, int>, TcConfig> g_cfg;  // (nacc, n) -> config; n = 0 is the default

TcConfig lookup_config(int nacc, int n) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  auto it = g_cfg.find({nacc, n});
  if (it != g_cfg.end()) return it->second;
  it = g_cfg.find({nacc, 0});
  if (it != g_cfg.end()) return it->second;
  TcConfig c;
  c.bk = 64;
  c.bn_cap = nacc == 1 ? 256 : 128;
  // real data on long axes: CTA pairs (each SM stages half of the S_k tile); measured on the
  // BF16X3 plane passes at n = 512: 0.299 ms against 0.321 ms for single CTAs
  c.pair = nacc == 1 && n >= 256;
  return c;
}

template <int NP, int NACC>
ts_status launch_pass(const __nv_bfloat16* A, const __nv_bfloat16* B, long long R, int n, EpiParams ep,
                      cudaStream_t s) {
  TcConfig c = lookup_config(NACC, n);
  if (2 * NACC * c.bn_cap > 512) c.bn_cap = 256 / NACC;  // two accumulator buffers must fit in TMEM
  if (c.bn_cap % 32 != 0) c.pair = false;
  // Fall back to a narrower K chunk, then a narrower N tile, until two stages fit.
  const int reserve = 1024 + 8 * (2 * MAX_STAGES + 6);
  for (;;) {
    const int bq = c.pair ? 32 : 16;
    int bn = ((n + bq - 1) / bq) * bq;
    if (bn > c.bn_cap) bn = c.bn_cap;
    const int stage = NACC * NP * BM * c.bk * 2 + NP * (c.pair ? bn / 2 : bn) * c.bk * 2;
    if ((SMEM_LIMIT - reserve) / stage >= 2) break;
    if (c.bk == 64)
      c.bk = 32;
    else if (c.bn_cap > 16)
      c.bn_cap /= 2;
    else
      break;
    if (c.bn_cap % 32 != 0) c.pair = false;
  }
  if (ep.out_mode == 0) {
  // one statement (a braced block), so that `if (c.bk == 32) TS_PAIR_DISPATCH(32, ..)` guards all of it
  #define TS_PAIR_DISPATCH(BKT, PO)                                                                 \
  {                                                                                                \
    if (c.pair) return launch_pass_t<NP, NACC, BKT, PO, true>(A, B, R, n, ep, c.bn_cap, s);       \
    return launch_pass_t<NP, NACC, BKT, PO, false>(A, B, R, n, ep, c.bn_cap, s);                  \
  }
    if (c.bk == 32) TS_PAIR_DISPATCH(32, true);
    TS_PAIR_DISPATCH(64, true);
  }
  if (c.bk == 32) TS_PAIR_DISPATCH(32, false);
  TS_PAIR_DISPATCH(64, false);
#undef TS_PAIR_DISPATCH
}

ts_status pass(int np, int nacc, const __nv_bfloat16* A, const __nv_bfloat16* B, long long R, int n,
               const EpiParams& ep, cudaStream_t s) {
  if (np == 1 && nacc == 1) return launch_pass<1, 1>(A, B, R, n, ep, s);
  if (np == 1 && nacc == 2) return launch_pass<1, 2>(A, B, R, n, ep, s);
  if (np == 2 && nacc == 1) return launch_pass<2, 1>(A, B, R, n, ep, s);
  if (np == 2 && nacc == 2) return launch_pass<2, 2>(A, B, R, n, ep, s);
  if (np == 3 && nacc == 1) return launch_pass<3, 1>(A, B, R, n, ep, s);
  return launch_pass<3, 2>(A, B, R, n, ep, s);
}

unsigned grid_1d(long long N) {
  long long g = (N + 255) / 256;
  if (g > 148 * 8) g = 148 * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

ts_status build_split_tables(ts_plan* p, ts_precision prec, cudaStream_t s) {
  const int np = bf16_planes(prec);
  if (np == 0) {
    set_error("precision %d is not implemented (available: TS_FP64, TS_BF16X1, TS_BF16X3, TS_BF16X6, TS_FP32)", (int)prec);
    return TS_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < p->d; ++k) {
    AxisTables* t = p->axis[k].get();
    std::lock_guard<std::mutex> lk(t->mu);
    if (!t->Bf[prec]) {
      const long long cnt = (long long)t->n * t->n;
      const long long padded = (long long)t->n * ((t->n + 7) & ~7);  // rows padded to 16 bytes
      __nv_bfloat16 *bf = nullptr, *bb = nullptr;
      TS_TRY(table_alloc((void**)&bf, sizeof(__nv_bfloat16) * np * padded, s));
      const ts_status st = table_alloc((void**)&bb, sizeof(__nv_bfloat16) * np * padded, s);
      if (st != TS_OK) {
        table_free(bf, t->device);
        return st;
      }
      TS_CHECK_CUDA(cudaMemsetAsync(bf, 0, sizeof(__nv_bfloat16) * np * padded, s));
      TS_CHECK_CUDA(cudaMemsetAsync(bb, 0, sizeof(__nv_bfloat16) * np * padded, s));
      // Forward: y_j = sum_i S[i][j] x_i, K-major operand B[j][i] = S[i][j]; backward:
      // y_i = sum_j St[j][i] x_j, operand B[i][j] = St[j][i] (for orthogonal tables St = S^T).
      k_split_table_t<<<grid_1d(cnt), 256, 0, s>>>(t->S, bf, t->n, np);
      k_split_table_t<<<grid_1d(cnt), 256, 0, s>>>(t->St, bb, t->n, np);
      TS_LAUNCHED(2);
      TS_CHECK_CUDA(cudaStreamSynchronize(s));  // published to other plans only once complete
      t->Bf[prec] = bf;
      t->Bb[prec] = bb;
      t->bytes += 2LL * np * padded * (long long)sizeof(__nv_bfloat16);
    }
    p->Bf[prec][k] = t->Bf[prec];
    p->Bb[prec][k] = t->Bb[prec];
  }
  return TS_OK;
}

namespace {

ts_status check_mixed(const ts_plan* p, ts_precision prec) {
  if (bf16_planes(prec) == 0) {
    set_error("precision %d is not implemented (available: TS_FP64, TS_BF16X1, TS_BF16X3, TS_BF16X6)", (int)prec);
    return TS_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < p->d; ++k) {
    if (p->N / p->n[k] >= (1LL << 31)) {
      set_error("split-precision path needs N/n_k < 2^31 (axis %d: n = %d)", k, p->n[k]);
      return TS_ERR_UNSUPPORTED;
    }
  }
  return TS_OK;
}

// Layout of a pass's plane output = the next pass's input (see EpiParams::on): rows of the
// next contracted axis, padded to a multiple of 8 elements.
void set_plane_output(EpiParams& ep, const ts_plan* p, int k) {
  if (p->d == 1) {  // one row: output column j is element j of the next input row
    ep.Ro = 1;
    ep.No = (p->n[0] + 7) & ~7;
    ep.on = ep.old = 1;
    return;
  }
  const int kn = (k + 1) % p->d;
  const long long R = p->N / p->n[k];
  ep.on = p->n[kn];
  ep.old = (p->n[kn] + 7) & ~7;
  ep.Ro = (R / ep.on) * ep.old;
  ep.No = (p->N / ep.on) * ep.old;
}

// The 2d contraction passes of one apply: planes in buf[0] -> ... -> `out` (out_mode of the
// last pass: 1 FP64 store, 2 complex128, 3 complex64, 4 FP64 accumulate), with the
// pointwise step fused into pass d-1.  emax_out (modes 1 / 4, may be NULL): raised to the
// largest biased exponent of the stored values (the caller zeroes it first).
// The epilogue of the last pass of an apply in a solve with a fixed-point iterate
// (out_mode 5-7, see EpiParams).
struct FixLast {
  FixScale fxs;
  int fix_in = 0, fix_out = 0;
  const long long* src = nullptr;
};

ts_status run_passes(const ts_plan* p, ts_precision prec, MixedOp op, double param, __nv_bfloat16* const buf[2],
                     const double2* tabs, const float2* tabsf, const int* tab_off, void* out, int last_mode,
                     cudaStream_t s, int* emax_out = nullptr, const FixLast* fix = nullptr) {
  const int np = bf16_planes(prec);
  const int nc = op == MixedOp::Exp ? 2 : 1;
  const int d = p->d;
  ts_status st = TS_OK;
  for (int t = 0; t < 2 * d && st == TS_OK; ++t) {
    const int k = t % d;
    const bool fwd = t < d;
    const bool last = t == 2 * d - 1;
    EpiParams ep{};
    ep.out_mode = last ? last_mode : 0;
    ep.out = last ? out : (void*)buf[(t + 1) & 1];
    ep.emax_out = last ? emax_out : nullptr;
    ep.scale_mode = 0;
    if (t == d - 1) {
      ep.scale_mode = op == MixedOp::Inverse ? 1 : 2;
      ep.sigma = op == MixedOp::Inverse ? param : 0.0;
      ep.rd = d - 1;
      for (int q = 0; q < d - 1; ++q) {
        ep.rn[q] = p->n[q];
        ep.rlam[q] = p->lam[q];
        ep.rph[q] = tabs ? tabs + tab_off[q] : nullptr;
      }
      ep.clam = p->lamf[k];
      ep.cph = tabsf ? tabsf + tab_off[k] : nullptr;
    }
    if (!last) set_plane_output(ep, p, k);
    if (last && fix) {
      ep.fxs = fix->fxs;
      ep.fix_in = fix->fix_in;
      ep.fix_out = fix->fix_out;
      ep.fix_src = fix->src;
    }
    const __nv_bfloat16* B = fwd ? p->Bf[prec][k] : p->Bb[prec][k];
    st = pass(np, nc, buf[t & 1], B, p->N / p->n[k], p->n[k], ep, s);
  }
  return st;
}

ts_status split_input(int np, ts_dtype dt, const void* in, __nv_bfloat16* planes, long long N, int n0,
                      cudaStream_t s, int* emax = nullptr) {
#define TS_SPLIT2(MODE, PAD)                                                               \
  (np == 1   ? k_split_input<1, MODE, PAD><<<grid_1d(N), 256, 0, s>>>(in, planes, N, n0, emax) \
   : np == 2 ? k_split_input<2, MODE, PAD><<<grid_1d(N), 256, 0, s>>>(in, planes, N, n0, emax) \
             : k_split_input<3, MODE, PAD><<<grid_1d(N), 256, 0, s>>>(in, planes, N, n0, emax))
#define TS_SPLIT(MODE) (n0 % 8 == 0 ? TS_SPLIT2(MODE, false) : TS_SPLIT2(MODE, true))
  if (dt == TS_R64 && n0 % 8 == 0 && N % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
      reinterpret_cast<uintptr_t>(planes) % 8 == 0) {
    if (np == 1)
      k_split_real4<1><<<grid_1d(N / 4), 256, 0, s>>>((const double*)in, planes, N, emax);
    else if (np == 2)
      k_split_real4<2><<<grid_1d(N / 4), 256, 0, s>>>((const double*)in, planes, N, emax);
    else
      k_split_real4<3><<<grid_1d(N / 4), 256, 0, s>>>((const double*)in, planes, N, emax);
  } else if (dt == TS_R64)
    TS_SPLIT(0);
  else if (dt == TS_C128)
    TS_SPLIT(1);
  else
    TS_SPLIT(2);
#undef TS_SPLIT
#undef TS_SPLIT2
  TS_LAUNCHED(1);
  return TS_OK;
}

}  // namespace

ts_status mixed_apply(const ts_plan* p, ts_precision prec, MixedOp op, double param, const void* in, void* out,
                      ts_dtype dt, cudaStream_t s) {
  TS_TRY(check_mixed(p, prec));
  const int np = bf16_planes(prec);
  const int nc = op == MixedOp::Exp ? 2 : 1;
  const long long N = p->N;
  const size_t plane_bytes = sizeof(__nv_bfloat16) * (size_t)nc * np * mixed_plane_elems(p);
  void *w0 = nullptr, *w1 = nullptr, *tabs = nullptr;
  TS_TRY(scratch_alloc(&w0, plane_bytes, s));
  ts_status st = scratch_alloc(&w1, plane_bytes, s);
  int tab_off[MAXD] = {};
  int tab_total = 0;
  if (st == TS_OK && op == MixedOp::Exp) {
    int tot = 0;
    for (int k = 0; k < p->d; ++k) {
      tab_off[k] = tot;
      tot += p->n[k];
    }
    tab_total = tot;
    st = scratch_alloc(&tabs, (sizeof(double2) + sizeof(float2)) * tot, s);
    for (int k = 0; k < p->d && st == TS_OK; ++k) {
      k_phase_table<<<(p->n[k] + 127) / 128, 128, 0, s>>>(p->lam[k], param, (double2*)tabs + tab_off[k],
                                                          (float2*)((double2*)tabs + tot) + tab_off[k], p->n[k]);
      count_launches(1);
      if (cudaGetLastError() != cudaSuccess) {
        set_error("phase table launch failed");
        st = TS_ERR_CUDA;
      }
    }
  }
  __nv_bfloat16* buf[2] = {(__nv_bfloat16*)w0, (__nv_bfloat16*)w1};
  if (st == TS_OK) st = split_input(np, dt, in, buf[0], N, p->n[0], s);
  if (st == TS_OK)
    st = run_passes(p, prec, op, param, buf, (const double2*)tabs,
                    tabs ? (const float2*)((const double2*)tabs + tab_total) : nullptr, tab_off, out,
                    dt == TS_R64 ? 1 : (dt == TS_C128 ? 2 : 3), s);
  scratch_free(w0, s);
  scratch_free(w1, s);
  scratch_free(tabs, s);
  return st;
}

namespace {

template <int NP, int NACC, int BKT, bool PO>
ts_status launch_list_t(const TcItemList& L, int smem, cudaStream_t s) {
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc_list<NP, NACC, BKT, PO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_LIMIT));
    attr_set = true;
  }
  if (g_num_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const unsigned grid = (unsigned)(L.total < g_num_sms ? L.total : g_num_sms);
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_rot_tc_list<NP, NACC, BKT, PO><<<grid, TC_THREADS, smem, s>>>(L);
  TS_LAUNCHED(1);
  if (tok) {
    // algorithmic work of all items: products x 2 R n^2 FLOP; planes in, planes or result out
    double flops = 0.0, bytes = 0.0;
    for (int i = 0; i < L.count; ++i) {
      const EpiParams& ep = L.item[i].ep;
      const double vals = (double)ep.R * ep.n;
      flops += 2.0 * Products<NP>::count * NACC * vals * ep.n;
      const double out_b = ep.out_mode == 0 ? 2.0 * NP * NACC
                         : ep.out_mode == 1 ? 8.0 : ep.out_mode == 2 ? 16.0 : ep.out_mode == 3 ? 8.0 : 16.0;
      bytes += vals * (2.0 * NP * NACC + out_b);
    }
    prof_end_launch(s, tok, PROF_TC_LIST, flops, bytes);
  }
  return TS_OK;
}

ts_status launch_list(int np, int nacc, int bk, bool po, const TcItemList& L, int smem, cudaStream_t s) {
#define TS_LIST_CASE(NP, NACC)                                                                            \
  if (np == NP && nacc == NACC) {                                                                         \
    if (bk == 64) return po ? launch_list_t<NP, NACC, 64, true>(L, smem, s) : launch_list_t<NP, NACC, 64, false>(L, smem, s); \
    return po ? launch_list_t<NP, NACC, 32, true>(L, smem, s) : launch_list_t<NP, NACC, 32, false>(L, smem, s);               \
  }
  TS_LIST_CASE(1, 1) TS_LIST_CASE(1, 2) TS_LIST_CASE(2, 1) TS_LIST_CASE(2, 2) TS_LIST_CASE(3, 1) TS_LIST_CASE(3, 2)
#undef TS_LIST_CASE
  set_error("no work-list kernel for %d planes, %d components", np, nacc);
  return TS_ERR_UNSUPPORTED;
}

}  // namespace

ts_status mixed_apply_batch(const BatchApply* q, int count, cudaStream_t s) {
  for (int i = 0; i < count; ++i) TS_TRY(check_mixed(q[i].p, q[i].prec));
  struct Work {
    __nv_bfloat16* buf[2] = {nullptr, nullptr};
    void* tabs = nullptr;
    int tab_off[MAXD] = {};
    int tab_total = 0;
    int np = 0, nc = 1;
  };
  std::vector<Work> w(count);
  ts_status st = TS_OK;
  int dmax = 0;
  // per item: plane buffers and (exp) phase tables
  for (int i = 0; i < count && st == TS_OK; ++i) {
    const ts_plan* p = q[i].p;
    w[i].np = bf16_planes(q[i].prec);
    w[i].nc = q[i].op == MixedOp::Exp ? 2 : 1;
    dmax = p->d > dmax ? p->d : dmax;
    const size_t plane_bytes = sizeof(__nv_bfloat16) * (size_t)w[i].nc * w[i].np * mixed_plane_elems(p);
    for (int b = 0; b < 2 && st == TS_OK; ++b) st = scratch_alloc((void**)&w[i].buf[b], plane_bytes, s);
    if (st == TS_OK && q[i].op == MixedOp::Exp) {
      int tot = 0;
      for (int k = 0; k < p->d; ++k) {
        w[i].tab_off[k] = tot;
        tot += p->n[k];
      }
      w[i].tab_total = tot;
      st = scratch_alloc(&w[i].tabs, (sizeof(double2) + sizeof(float2)) * tot, s);
      for (int k = 0; k < p->d && st == TS_OK; ++k) {
        k_phase_table<<<(p->n[k] + 127) / 128, 128, 0, s>>>(p->lam[k], q[i].param,
                                                            (double2*)w[i].tabs + w[i].tab_off[k],
                                                            (float2*)((double2*)w[i].tabs + tot) + w[i].tab_off[k],
                                                            p->n[k]);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) {
          set_error("phase table launch failed");
          st = TS_ERR_CUDA;
        }
      }
    }
  }
  // input split: one launch per plane count over all its items
  for (int np = 1; np <= 3 && st == TS_OK; ++np) {
    std::vector<int> idx;
    for (int i = 0; i < count; ++i)
      if (w[i].np == np) idx.push_back(i);
    for (size_t c0 = 0; c0 < idx.size() && st == TS_OK; c0 += TC_LIST_MAX) {
      SplitList L{};
      int blocks = 0;
      for (size_t c = c0; c < idx.size() && c < c0 + TC_LIST_MAX; ++c) {
        const int i = idx[c];
        SplitItem& it = L.item[L.count++];
        it.in = q[i].in;
        it.planes = w[i].buf[0];
        it.N = q[i].p->N;
        it.n0 = q[i].p->n[0];
        it.mode = q[i].dt == TS_R64 ? 0 : (q[i].dt == TS_C128 ? 1 : 2);
        it.block_begin = blocks;
        long long nb = (it.N + 255) / 256;
        blocks += (int)(nb < 148 * 4 ? nb : 148 * 4);
      }
      if (np == 1) k_split_list<1><<<blocks, 256, 0, s>>>(L);
      else if (np == 2) k_split_list<2><<<blocks, 256, 0, s>>>(L);
      else k_split_list<3><<<blocks, 256, 0, s>>>(L);
      TS_LAUNCHED(1);
    }
  }
  // the 2d passes: pass st of every item that has one, one launch per (planes, components,
  // planes-out) group and up to TC_LIST_MAX items
  const int reserve = 1024 + 8 * (2 * MAX_STAGES + 6);
  for (int stage = 0; stage < 2 * dmax && st == TS_OK; ++stage) {
    std::map<std::tuple<int, int, bool>, std::vector<int>> groups;
    for (int i = 0; i < count; ++i) {
      const int d = q[i].p->d;
      if (stage < 2 * d) groups[std::make_tuple(w[i].np, w[i].nc, stage != 2 * d - 1)].push_back(i);
    }
    for (auto& gkv : groups) {
      const int np = std::get<0>(gkv.first), nacc = std::get<1>(gkv.first);
      const bool po = std::get<2>(gkv.first);
      const std::vector<int>& idx = gkv.second;
      for (size_t c0 = 0; c0 < idx.size() && st == TS_OK; c0 += TC_LIST_MAX) {
        const size_t c1 = idx.size() < c0 + TC_LIST_MAX ? idx.size() : c0 + TC_LIST_MAX;
        const int cap = nacc == 1 ? 256 : 128;  // two accumulator buffers fit in TMEM
        int bn_max = 16;
        for (size_t c = c0; c < c1; ++c) {
          const ts_plan* p = q[idx[c]].p;
          int bn = ((p->n[stage % p->d] + 15) / 16) * 16;
          bn = bn > cap ? cap : bn;
          bn_max = bn > bn_max ? bn : bn_max;
        }
        int bk = 64;
        auto stage_bytes = [&](int b) { return nacc * np * BM * b * 2 + np * bn_max * b * 2; };
        if ((SMEM_LIMIT - reserve) / stage_bytes(64) < 2) bk = 32;
        int ns = (SMEM_LIMIT - reserve) / stage_bytes(bk);
        ns = ns > MAX_STAGES ? MAX_STAGES : ns;
        if (ns < 2) {
          set_error("work-list tile does not fit in shared memory");
          st = TS_ERR_UNSUPPORTED;
          break;
        }
        TcItemList L{};
        L.bn_max = bn_max;
        L.nstages = ns;
        long long units = 0;
        for (size_t c = c0; c < c1 && st == TS_OK; ++c) {
          const int i = idx[c];
          const ts_plan* p = q[i].p;
          const int d = p->d, k = stage % d;
          const bool fwd = stage < d, last = stage == 2 * d - 1;
          const int n = p->n[k];
          const long long R = p->N / n;
          TcItem& it = L.item[L.count++];
          EpiParams& ep = it.ep;
          ep = EpiParams{};
          ep.out_mode = last ? (q[i].dt == TS_R64 ? 1 : (q[i].dt == TS_C128 ? 2 : 3)) : 0;
          ep.out = last ? q[i].out : (void*)w[i].buf[(stage + 1) & 1];
          if (stage == d - 1) {
            ep.scale_mode = q[i].op == MixedOp::Inverse ? 1 : 2;
            ep.sigma = q[i].op == MixedOp::Inverse ? q[i].param : 0.0;
            ep.rd = d - 1;
            for (int j = 0; j < d - 1; ++j) {
              ep.rn[j] = p->n[j];
              ep.rlam[j] = p->lam[j];
              ep.rph[j] = w[i].tabs ? (const double2*)w[i].tabs + w[i].tab_off[j] : nullptr;
            }
            ep.clam = p->lamf[k];
            ep.cph = w[i].tabs ? (const float2*)((const double2*)w[i].tabs + w[i].tab_total) + w[i].tab_off[k]
                               : nullptr;
          }
          int bn = ((n + 15) / 16) * 16;
          bn = bn > cap ? cap : bn;
          ep.R = R;
          ep.n = n;
          ep.N = p->N;
          if (last) {
            ep.Ro = R;
            ep.No = p->N;
            ep.on = ep.old = 1;
          } else {
            set_plane_output(ep, p, k);
          }
          ep.bn = bn;
          ep.nstages = ns;
          const __nv_bfloat16* B = fwd ? p->Bf[q[i].prec][k] : p->Bb[q[i].prec][k];
          st = make_map(&it.tmA, w[i].buf[stage & 1], n, R, nacc * np, bk, BM);
          if (st == TS_OK) st = make_map(&it.tmB, B, n, n, np, bk, bn);
          it.mtiles = (int)((R + BM - 1) / BM);
          it.ntiles = (n + bn - 1) / bn;
          it.nk = (n + bk - 1) / bk;
          it.unit_begin = units;
          units += (long long)it.mtiles * it.ntiles;
        }
        L.total = units;
        if (st == TS_OK) st = launch_list(np, nacc, bk, po, L, ns * stage_bytes(bk) + reserve, s);
      }
    }
  }
  for (int i = 0; i < count; ++i) {
    scratch_free(w[i].buf[0], s);
    scratch_free(w[i].buf[1], s);
    scratch_free(w[i].tabs, s);
  }
  return st;
}

ts_status mixed_inverse_buffers(const ts_plan* p, ts_precision prec, double sigma, const double* b, double* u,
                                __nv_bfloat16* w0, __nv_bfloat16* w1, cudaStream_t s) {
  TS_TRY(check_mixed(p, prec));
  __nv_bfloat16* buf[2] = {w0, w1};
  TS_TRY(split_input(bf16_planes(prec), TS_R64, b, buf[0], p->N, p->n[0], s));
  return run_passes(p, prec, MixedOp::Inverse, sigma, buf, nullptr, nullptr, nullptr, u, 1, s);
}

ts_status mixed_refine(const ts_plan* p, ts_precision prec, double sigma, const double* b, double* u,
                       int refinements, cudaStream_t s) {
  ts_precision sched[17];
  for (int k = 0; k <= refinements && k < 17; ++k) sched[k] = prec;
  return mixed_solve_schedule(p, sched, refinements + 1, sigma, b, u, s);
}

namespace {

// Whether a refined solve on plan p can carry its iterate as the fixed-point integer
// U = u 2^s (d = 3, one spacing h, the exact folded residual applies, axis-0 rows of an
// even length and b 16-byte aligned for the residual's TMA tiles), and the factor beta of a
// bound max|u| <= beta max|b|: 1 / (sigma + min V1) when that is positive (A is then an
// M-matrix with A 1 >= (sigma + min V1) 1, so ||A^{-1}||_inf <= 1 / (sigma + min V1)), and
// sqrt(N) / lambda_min(A) from the 2-norm.  The scale of U_0 follows from that bound, so it
// may be loose by beta ||A||_inf (max|u| >= max|b| / ||A||_inf): at most 2^24 is accepted,
// which leaves U_0 above 30 significant bits.  *l2b = ceil(log2 beta) + 2.
bool fix_iterate_bound(const ts_plan* p, double sigma, const double* b, int* l2b) {
  if (p->d != 3 || !isotropic_h(p) || p->n[0] % 2 != 0) return false;
  if (reinterpret_cast<uintptr_t>(b) % 16 != 0) return false;
  double fmin = 0.0, fmax = 0.0, lmin = sigma;
  for (int k = 0; k < 3; ++k) {
    const std::vector<double>& f = p->axis[k]->f;
    const std::vector<double>& lam = p->axis[k]->lam_host;
    if (f.empty() || lam.empty()) return false;
    double lo = f[0], hi = std::fabs(f[0]);
    for (double v : f) {
      lo = v < lo ? v : lo;
      hi = std::fabs(v) > hi ? std::fabs(v) : hi;
    }
    fmin += lo;
    fmax += hi;
    lmin += lam[0];
  }
  const double h = 2.0 * p->L[0] / (p->n[0] + 1);
  const double anorm = 12.0 / (h * h) + std::fabs(sigma) + fmax;
  double beta = HUGE_VAL;
  if (sigma + fmin > 0.0) beta = 1.0 / (sigma + fmin);
  if (lmin > 0.0) beta = std::fmin(beta, std::sqrt((double)p->N) / lmin);
  if (!std::isfinite(beta) || !(std::log2(beta * anorm) <= 24.0)) return false;
  *l2b = (int)std::ceil(std::log2(beta)) + 2;
  return true;
}

}  // namespace

ts_status mixed_solve_schedule(const ts_plan* p, const ts_precision* sched, int count, double sigma,
                               const double* b, double* u, cudaStream_t s) {
  int npmax = 0;
  for (int k = 0; k < count; ++k) {
    TS_TRY(check_mixed(p, sched[k]));
    npmax = bf16_planes(sched[k]) > npmax ? bf16_planes(sched[k]) : npmax;
  }
  const int refinements = count - 1;
  const long long N = p->N;
  const size_t plane_bytes = sizeof(__nv_bfloat16) * (size_t)npmax * mixed_plane_elems(p);
  int l2b = 0;
  const bool fix_iter = refinements > 0 && fix_iterate_bound(p, sigma, b, &l2b);
  void *w0 = nullptr, *w1 = nullptr, *partial = nullptr, *qtab = nullptr, *ubuf = nullptr;
  TS_TRY(scratch_alloc(&w0, plane_bytes, s));
  ts_status st = scratch_alloc(&w1, plane_bytes, s);
  if (st == TS_OK) st = scratch_alloc(&partial, sizeof(double) * 2 * RED_BLOCKS, s);
  if (st == TS_OK && qtable_count(p) > 0 && refinements > 0)
    st = scratch_alloc(&qtab, sizeof(long long) * qtable_count(p), s);
  __nv_bfloat16* buf[2] = {(__nv_bfloat16*)w0, (__nv_bfloat16*)w1};
  // The fixed-point iterate: u_0 is stored as U_0 = u_0 2^s0 (int64), every refinement adds
  // its correction to U in integer arithmetic (exact), the residuals read U directly, and
  // the last refinement writes the FP64 u = U 2^-s.
  FixedOperator fo;
  if (st == TS_OK && fix_iter) st = fixed_operator_prepare(p, sigma, (long long*)qtab, &fo, s);
  if (st == TS_OK && fix_iter && fo.ok) {
    st = scratch_alloc(&ubuf, sizeof(long long) * (size_t)N, s);
    int* fx = (int*)partial;  // fx[0] = emax of b, fx[1] = emax of u_0
    if (st == TS_OK && cudaMemsetAsync(fx, 0, 2 * sizeof(int), s) != cudaSuccess) {
      set_error("memset failed");
      st = TS_ERR_CUDA;
    }
    FixLast fl;
    fl.fxs.fx = fx;
    fl.fxs.hu = fo.H;
    fl.fxs.l2b = l2b;
    long long* U = (long long*)ubuf;
    if (st == TS_OK) st = split_input(bf16_planes(sched[0]), TS_R64, b, buf[0], N, p->n[0], s, fx);
    fl.fix_out = 0;
    if (st == TS_OK)
      st = run_passes(p, sched[0], MixedOp::Inverse, sigma, buf, nullptr, nullptr, nullptr, U, 5, s, fx + 1, &fl);
    for (int it = 0; it < refinements && st == TS_OK; ++it) {
      const bool last = it + 1 == refinements;
      const ts_precision prec = sched[it + 1];
      st = residual_fixu(p, U, b, fo.qtab, fo.F, fl.fxs, it == 0 ? 0 : 1, buf[0], bf16_planes(prec), s);
      fl.fix_in = it == 0 ? 0 : 1;
      fl.fix_out = 1;
      fl.src = U;
      if (st == TS_OK)
        st = run_passes(p, prec, MixedOp::Inverse, sigma, buf, nullptr, nullptr, nullptr, last ? (void*)u : (void*)U,
                        last ? 7 : 6, s, nullptr, &fl);
    }
  } else if (st == TS_OK) {
    // On isotropic grids the residual's Laplacian is summed in exact fixed point, scaled by
    // the largest exponent of u; the pass that writes u finds it on the way out.
    const bool fixed = isotropic_h(p);
    int* emax = (int*)partial;
    auto zero_emax = [&]() -> ts_status {
      if (fixed && cudaMemsetAsync(emax, 0, sizeof(int), s) != cudaSuccess) {
        set_error("memset failed");
        return TS_ERR_CUDA;
      }
      return TS_OK;
    };
    // u_0 = P_0 b
    st = split_input(bf16_planes(sched[0]), TS_R64, b, buf[0], N, p->n[0], s);
    if (st == TS_OK && refinements > 0) st = zero_emax();
    if (st == TS_OK)
      st = run_passes(p, sched[0], MixedOp::Inverse, sigma, buf, nullptr, nullptr, nullptr, u, 1, s,
                      fixed && refinements > 0 ? emax : nullptr);
    // u_{k+1} = u_k + P_{k+1} (b - A u_k), residual in FP64, split straight into the planes
    for (int it = 0; it < refinements && st == TS_OK; ++it) {
      const bool more = it + 1 < refinements;
      const ts_precision prec = sched[it + 1];
      const int np = bf16_planes(prec);
      if (fixed)
        st = residual_split_fixed(p, sigma, u, b, buf[0], np, emax, (long long*)qtab, s);
      else
        st = stencil_residual_split(p, nullptr, sigma, u, b, buf[0], np, (double*)partial, s);
      if (st == TS_OK && more) st = zero_emax();
      if (st == TS_OK)
        st = run_passes(p, prec, MixedOp::Inverse, sigma, buf, nullptr, nullptr, nullptr, u, 4, s,
                        fixed && more ? emax : nullptr);
    }
  }
  scratch_free(w0, s);
  scratch_free(w1, s);
  scratch_free(partial, s);
  scratch_free(qtab, s);
  scratch_free(ubuf, s);
  return st;
}

ts_status tc_prepare_kernels() {
  // Shared-memory opt-in for every instantiation, outside any stream capture.
#define TS_PREP1(NP, NACC, BKT, PO, PAIR)                                                              \
  TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc<NP, NACC, BKT, PO, PAIR>,                                \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT))
#define TS_PREP(NP, NACC, BKT, PO) TS_PREP1(NP, NACC, BKT, PO, false); TS_PREP1(NP, NACC, BKT, PO, true)
  TS_PREP(1, 1, 64, true); TS_PREP(1, 1, 64, false); TS_PREP(1, 1, 32, true); TS_PREP(1, 1, 32, false);
  TS_PREP(1, 2, 64, true); TS_PREP(1, 2, 64, false); TS_PREP(1, 2, 32, true); TS_PREP(1, 2, 32, false);
  TS_PREP(2, 1, 64, true); TS_PREP(2, 1, 64, false); TS_PREP(2, 1, 32, true); TS_PREP(2, 1, 32, false);
  TS_PREP(2, 2, 64, true); TS_PREP(2, 2, 64, false); TS_PREP(2, 2, 32, true); TS_PREP(2, 2, 32, false);
  TS_PREP(3, 1, 64, true); TS_PREP(3, 1, 64, false); TS_PREP(3, 1, 32, true); TS_PREP(3, 1, 32, false);
  TS_PREP(3, 2, 64, true); TS_PREP(3, 2, 64, false); TS_PREP(3, 2, 32, true); TS_PREP(3, 2, 32, false);
#undef TS_PREP1
#undef TS_PREP
#define TS_PREPL(NP, NACC)                                                                                     \
  TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc_list<NP, NACC, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT)); \
  TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc_list<NP, NACC, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT)); \
  TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc_list<NP, NACC, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT)); \
  TS_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc_list<NP, NACC, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT))
  TS_PREPL(1, 1); TS_PREPL(1, 2); TS_PREPL(2, 1); TS_PREPL(2, 2); TS_PREPL(3, 1); TS_PREPL(3, 2);
#undef TS_PREPL
  if (g_num_sms == 0) {
    int dev = 0;
    TS_CHECK_CUDA(cudaGetDevice(&dev));
    TS_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return TS_OK;
}

ts_status tc_config_set(int complex_data, int n, int bk, int bn_cap, int cluster) {
  if (bk == 0 && bn_cap == 0 && cluster == 0 && n >= 0) {  // forget: back to the built-in choice
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg.erase({complex_data ? 2 : 1, n});
    return TS_OK;
  }
  if ((bk != 32 && bk != 64) || bn_cap < 16 || bn_cap > 256 || bn_cap % 16 != 0 || n < 0 ||
      (cluster != 1 && cluster != TS_TC_PAIR)) {
    set_error("invalid tensor-core tile configuration (bk %d, bn_cap %d, cluster %d; cluster is 1 or TS_TC_PAIR)",
              bk, bn_cap, cluster);
    return TS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  TcConfig c;
  c.bk = bk;
  c.bn_cap = bn_cap;
  c.pair = cluster == TS_TC_PAIR;
  g_cfg[{complex_data ? 2 : 1, n}] = c;
  return TS_OK;
}

namespace {
// One thread waits, with the kernels' bounded wait, on a barrier that nothing arrives on;
// after `cycles` clocks the wait gives up, records code 9 and the kernel returns.
__global__ void k_wait_selftest(long long cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  tc::fence_barrier_init();
  if (tc::mbar_try_wait(&bar, 0)) return;
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(&bar, 0)) {
    if (clock64() - t0 > cycles) {
      atomicExch(&g_tc_error, 9);
      return;
    }
  }
}
}  // namespace

ts_status wait_selftest(long long cycles, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(cycles);
  TS_LAUNCHED(1);
  return TS_OK;
}

ts_status mixed_error_flag(int* host_flag, bool reset, cudaStream_t s) {
  TS_CHECK_CUDA(cudaMemcpyFromSymbolAsync(host_flag, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (reset) {
    int zero = 0;
    TS_CHECK_CUDA(cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  }
  return TS_OK;
}

}  // namespace ts
