// FP64 mode-k contraction in rotating form (steps 2 and 4 of Sec. 2.1, one axis).
//
// The grid function X, whose fastest axis is the one being contracted (length n), is
// viewed as a row-major matrix X[r][i], r < R = N/n.  One pass computes
//     Y[r + R*j] = sum_i X[r][i] * B[i][j]
// i.e. Y = (X B)^T stored with r fastest: the contracted axis moves to the slowest
// position, so d passes visit every axis once and return the original axis order.
// Forward transform: B = S_k (B[i][j] = S_k[i][j]); backward: B = S_k^T.
// Complex data (ncomp = 2, interleaved) is a real GEMM with M = 2R rows m = 2r + c,
// because S_k is real: element (r, i, c) sits at 2(r n + i) + c, output (m, j) at m + 2R j.
//
// On B300 FP64 runs on the FFMA64 pipe (about 1.1 TFLOP/s measured; the m8n8k4 DMMA
// path measured lower), so this kernel is a plain register-tiled SIMT GEMM: a 256-thread
// CTA computes a BM x BN output tile, each thread a 4 x 4 micro-tile, with the K loop
// staged through shared memory in chunks of BK.  Out-of-range rows/columns/K are
// zero-filled on load and skipped on store, so any n and R are accepted.
#include "common.cuh"

namespace ts {
namespace {

template <int BN, int BK, int NC>
__global__ void __launch_bounds__(256) k_rot_fp64(const double* __restrict__ X, double* __restrict__ Y,
                                                  const double* __restrict__ B, long long R, int n) {
  constexpr int TM = 4, TN = 4;
  constexpr int NCOLG = BN / TN;
  constexpr int NROWG = 256 / NCOLG;
  constexpr int BM = NROWG * TM;
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  const long long M = R * NC;
  const long long m0 = (long long)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tm = tid % NROWG, tn = tid / NROWG;
  double acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.0;

  for (int k0 = 0; k0 < n; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int mm, kk;
      if (NC == 1) {
        mm = e / BK;
        kk = e % BK;
      } else {
        int rr = e / (2 * BK), w = e % (2 * BK);
        kk = w >> 1;
        mm = 2 * rr + (w & 1);
      }
      long long m = m0 + mm;
      int k = k0 + kk;
      double v = 0.0;
      if (m < M && k < n) {
        long long r = m / NC;
        int c = (int)(m - r * NC);
        v = X[(r * n + k) * NC + c];
      }
      As[kk][mm] = v;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk = e / BN, nn = e % BN;
      int k = k0 + kk, j = j0 + nn;
      Bs[kk][nn] = (k < n && j < n) ? B[(long long)k * n + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[kk][tm * TM + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[kk][tn * TN + q];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < TN; ++y) {
    int j = j0 + tn * TN + y;
    if (j >= n) continue;
#pragma unroll
    for (int x = 0; x < TM; ++x) {
      long long m = m0 + tm * TM + x;
      if (m < M) Y[m + M * j] = acc[x][y];
    }
  }
}

template <int BN, int BK, int NC>
ts_status launch(const double* X, double* Y, const double* B, long long R, int n, cudaStream_t s) {
  constexpr int BM = (256 / (BN / 4)) * 4;
  long long M = R * NC;
  long long gx = (M + BM - 1) / BM;
  TS_REQUIRE(gx < (1LL << 31), "rot_pass_fp64: grid too large (M=%lld)", M);
  dim3 grid((unsigned)gx, (unsigned)((n + BN - 1) / BN));
  void* tok = nullptr;
  if (prof_enabled()) prof_begin_launch(s, &tok);
  k_rot_fp64<BN, BK, NC><<<grid, 256, 0, s>>>(X, Y, B, R, n);
  TS_LAUNCHED(1);
  if (tok) prof_end_launch(s, tok, PROF_FP64_PASS, 2.0 * (double)M * n * n, 16.0 * (double)M * n);
  return TS_OK;
}

template <int NC>
ts_status dispatch(const double* X, double* Y, const double* B, long long R, int n, cudaStream_t s) {
  if (n <= 8) return launch<8, 8, NC>(X, Y, B, R, n, s);
  if (n <= 16) return launch<16, 16, NC>(X, Y, B, R, n, s);
  if (n <= 32) return launch<32, 16, NC>(X, Y, B, R, n, s);
  return launch<64, 16, NC>(X, Y, B, R, n, s);
}

}  // namespace

ts_status rot_pass_fp64(const double* X, double* Y, const double* B, long long R, int n, int ncomp,
                        cudaStream_t s) {
  if (ncomp == 1) return dispatch<1>(X, Y, B, R, n, s);
  return dispatch<2>(X, Y, B, R, n, s);
}

}  // namespace ts
