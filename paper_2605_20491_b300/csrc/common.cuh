// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tschrod.h"

namespace ts {

constexpr int MAXD = TS_MAX_DIM;
constexpr int NPREC = 7;
constexpr int MAX_PLANES = 3;

// Thread-local error message of the last failing call.
void set_error(const char* fmt, ...);
void clear_error();

#define TS_CHECK_CUDA(call)                                                               \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      ::ts::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,                  \
                      cudaGetErrorString(_e));                                            \
      return _e == cudaErrorMemoryAllocation ? TS_ERR_NO_MEMORY : TS_ERR_CUDA;            \
    }                                                                                     \
  } while (0)

// Every kernel launch of the library goes through TS_LAUNCHED(count): it adds to the
// process-wide launch counter (ts_launch_count) and checks the launch.
void count_launches(int k);
#define TS_LAUNCHED(k)                       \
  do {                                       \
    ::ts::count_launches(k);                 \
    TS_CHECK_CUDA(cudaGetLastError());       \
  } while (0)

// Live per-kernel timing (ts_profile_begin / ts_profile_end): when enabled, the launch
// sites of the contraction kernels bracket each launch with CUDA events on its stream.
enum ProfKind {
  PROF_TC_PASS = 0,      // split-precision tensor-core pass writing 2 or 3 bf16 planes
  PROF_FP64_PASS = 1,
  PROF_SMALL_PASS = 2,
  PROF_RESIDUAL = 3,
  PROF_TC_PASS_X1 = 4,   // the same kernel writing one bf16 plane (BF16X1)
  PROF_TC_PASS_OUT = 5,  // the same kernel writing the FP64 / complex result (last pass, any planes)
  PROF_TC_LIST = 6,      // the work-list form of the pass (batched applies)
  PROF_NKINDS = 7
};
bool prof_enabled();
void prof_begin_launch(cudaStream_t s, void** token);
void prof_end_launch(cudaStream_t s, void* token, int kind, double flops, double bytes);

#define TS_TRY(expr)                       \
  do {                                     \
    ts_status _s = (expr);                 \
    if (_s != TS_OK) return _s;            \
  } while (0)

#define TS_REQUIRE(cond, ...)              \
  do {                                     \
    if (!(cond)) {                         \
      ::ts::set_error(__VA_ARGS__);        \
      return TS_ERR_INVALID_ARG;           \
    }                                      \
  } while (0)

// Per-axis parameters passed by value to pointwise kernels.
struct AxisParams {
  int d;
  int n[MAXD];
  long long stride[MAXD];   // stride of axis k in vec() order
  double ih2[MAXD];         // 1 / h_k^2
  const double* tab[MAXD];  // per-axis table (eigenvalues or potential samples), n[k] entries
};

}  // namespace ts

namespace ts {

// Device tables of one axis: the eigendecomposition of H_k = M^{-1} Stiff + diag f (Q^1:
// h^-2 tridiag(-1,2,-1) + diag f) and the copies derived from it.  Shared by every plan (and
// every request) whose axis has the same (n, L, f, order, frame) on the same device; freed
// when the last user lets go of it.
//
// S and St are the operands of the forward and backward contractions in the rotating form
// Y = X^T B (y_j = sum_i B[i][j] x_i): S = (T^{-1})^T = M^{1/2} Q and St = T^T = Q^T M^{-1/2}.
// For Q^1 (M = h I, the h^{+-1/2} cancel) and in the symmetric frame (the frame of PCG for
// Q^k, where the unknown is M^{1/2} u) they are Q and Q^T.
struct AxisTables {
  int device = 0;
  int n = 0;
  double L = 0.0;
  int order = 1;                     // the k of Q^k
  int frame = 0;                     // Q^k: 0 = the plan's own unknowns, 1 = M^{1/2} u
  std::vector<double> f;             // host copy of the samples (cache key)
  void* block = nullptr;             // one allocation: S, St, lam, f, lamf (+ band, mh, mhi)
  double* S = nullptr;               // forward operand S[i][j], see above
  double* St = nullptr;              // backward operand
  double* lam = nullptr;             // eigenvalues, ascending
  double* fdev = nullptr;            // potential samples
  float* lamf = nullptr;             // eigenvalues rounded to FP32
  // Split bf16 planes per precision, [plane][n][n]: S^T (forward operand, Bf) and S
  // (backward operand, Bb), contracted index contiguous (K-major tensor-core operands).
  __nv_bfloat16* Bf[NPREC] = {};
  __nv_bfloat16* Bb[NPREC] = {};
  float* Sf32 = nullptr;             // S and S^T rounded to FP32 (small-n path)
  float* Stf32 = nullptr;
  // Q^k, k >= 2: the 1D Laplacian as a band, band[i * (2k+1) + o] = K[i][i + o - k] (zero
  // outside [0, n)), with K = M^{-1} Stiff (frame 0) or M^{-1/2} Stiff M^{-1/2} (frame 1);
  // mh = M^{1/2} and mhi = M^{-1/2} (diagonals).
  double* band = nullptr;
  double* mh = nullptr;
  double* mhi = nullptr;
  std::vector<double> lam_host, S_host;  // S_host: T = M^{-1/2} Q, the eigenvectors of H_k
  long long bytes = 0;
  std::mutex mu;                     // guards the lazily built precision copies
  ~AxisTables();
};

}  // namespace ts

// The plan: per-axis device tables (pointers into shared AxisTables).
struct ts_plan {
  int device = 0;
  int d = 0;
  int n[TS_MAX_DIM] = {};
  double L[TS_MAX_DIM] = {};
  long long N = 0;
  int nmax = 0;
  unsigned precision_mask = 1u;
  std::shared_ptr<ts::AxisTables> axis[TS_MAX_DIM];
  double* S[TS_MAX_DIM] = {};
  double* St[TS_MAX_DIM] = {};
  double* lam[TS_MAX_DIM] = {};
  float* lamf[TS_MAX_DIM] = {};
  float* Sf32[TS_MAX_DIM] = {};
  float* Stf32[TS_MAX_DIM] = {};
  double* f[TS_MAX_DIM] = {};
  __nv_bfloat16* Bf[ts::NPREC][TS_MAX_DIM] = {};
  __nv_bfloat16* Bb[ts::NPREC][TS_MAX_DIM] = {};
  long long bytes = 0;
  // Q^k, k >= 2 (order 1 leaves these empty)
  int order = 1;
  const double* band[TS_MAX_DIM] = {};  // banded K_k of this plan's frame, 2 * order + 1 per row
  const double* mh[TS_MAX_DIM] = {};    // M_k^{1/2}
  const double* mhi[TS_MAX_DIM] = {};   // M_k^{-1/2}
  ts_plan* sym = nullptr;               // the same grid in the frame M^{1/2} u (owned), or NULL
  ts_plan() = default;
  ts_plan(const ts_plan&) = delete;
  ts_plan& operator=(const ts_plan&) = delete;
  ~ts_plan();
};

namespace ts {

// Plans whose 1D operators are not the Q^1 tridiagonal: Q^k (k >= 2) and Hermite (order -1).
// They carry a band table, M^{+-1/2} and a symmetric twin.
inline bool banded_plan(const ts_plan* p) { return p->order >= 2 || p->order == -1; }
// Half-width of axis k's band: k of Q^k, n_k - 1 (dense) for Hermite.
inline int band_halfwidth(const ts_plan* p, int k) { return p->order == -1 ? p->n[k] - 1 : p->order; }

// Device-side helpers implemented in the .cu files.
AxisParams axis_params(const ts_plan* p, bool eig_tables);

// Scratch allocation from the stream-ordered pool.
ts_status scratch_alloc(void** ptr, size_t bytes, cudaStream_t s);
// Configure that pool for the current device now (outside any graph capture).
void scratch_pool_prepare();
void scratch_free(void* ptr, cudaStream_t s);

// Device memory of the resident per-axis tables: stream-ordered allocations from a
// per-device pool that keeps its memory mapped (release threshold unbounded), so that
// creating and evicting tables never synchronises the device (cudaMalloc/cudaFree would
// wait for every kernel in flight, serialising plan builders against the GPU work of
// earlier requests).  table_free requires that no enqueued work still reads the block.
ts_status table_alloc(void** ptr, size_t bytes, cudaStream_t s);
void table_free(void* ptr, int device);

// Eigendecomposition of a symmetric tridiagonal matrix on the host (implicit QR with the
// Wilkinson shift): lam ascending, Z column-major n x n.  False if it did not converge.
bool tridiag_eig_host(int n, const double* diag, const double* offdiag, double* lam, double* Z);
constexpr int TRIDIAG_HOST_MAX = 192;  // Q^1 axes up to this length use it in plan builds

// FP64 contraction pass (rotating form): see mode_fp64.cu.
ts_status rot_pass_fp64(const double* X, double* Y, const double* B, long long R, int n, int ncomp,
                        cudaStream_t s);
// Pointwise kernels: see pointwise.cu.
ts_status scale_inverse_fp64(const ts_plan* p, double sigma, double* X, cudaStream_t s);
ts_status scale_exp_c128(const ts_plan* p, double tau, double* X, cudaStream_t s);
ts_status phase_v2_c128(long long N, const double* V2, double theta_scale, double* psi, cudaStream_t s);
ts_status phase_v2_c64(long long N, const double* V2, double theta_scale, float* psi, cudaStream_t s);
ts_status convert_c64_to_c128(long long N, const float* in, double* out, cudaStream_t s);
ts_status convert_c128_to_c64(long long N, const double* in, float* out, cudaStream_t s);

// Drivers: see apply.cu.
ts_status apply_inverse_impl(const ts_plan* p, double sigma, const double* b, double* u,
                             ts_precision prec, cudaStream_t s);
ts_status apply_exp_impl(const ts_plan* p, double tau, const void* in, void* out, ts_dtype dt,
                         ts_precision prec, cudaStream_t s);

}  // namespace ts
