// ts_apply_inverse_noalloc: the direct inverse apply of ts_apply_inverse, with its work
// buffers taken from a fixed array compiled into the library instead of from the CUDA
// memory pool.
//
// Who needs it: callers that must not allocate device memory while they run -- a host
// application that hands the whole device to its own allocator up front, or a
// latency-critical loop that cannot afford cudaMalloc/cudaFree (cudaFree synchronises the
// device) or a stream-ordered pool that may have to grow.  Such callers still own and
// pass the input and output arrays; only the two intermediate buffers live here.
//
// The scratch is one file-scope __device__ array of NOALLOC_SCRATCH_BYTES (32 MiB).  Every
// GPU that loads this library holds a copy of it until the process exits.  All calls on a
// device share it and it keeps whatever the last call left there; nothing in it needs to
// start at zero (every pass overwrites what it later reads).  Calls whose execution
// overlaps on the GPU (different streams, or different host threads) race on the array
// and give wrong results: serialise them.
#include <mutex>

#include "common.cuh"
#include "mixed.cuh"

namespace ts {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_addr_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  The first call on each
// device resolves it with cudaGetSymbolAddress (that device must be current); later calls
// reuse the cached address.
ts_status scratch_address(void** out) {
  int dev = 0;
  TS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device ordinal %d out of range for the no-allocation scratch", dev);
    return TS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
      return TS_ERR_CUDA;
    }
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return TS_OK;
}

// The FP64 inverse apply (steps 2-4 of Sec. 2.1) on caller-provided work buffers.
ts_status fp64_inverse_buffers(const ts_plan* p, double sigma, const double* b, double* u, double* w0, double* w1,
                               cudaStream_t s) {
  const long long N = p->N;
  double* buf[2] = {w0, w1};
  const double* src = b;
  int cur = 0;
  for (int k = 0; k < p->d; ++k) {
    TS_TRY(rot_pass_fp64(src, buf[cur], p->S[k], N / p->n[k], p->n[k], 1, s));
    src = buf[cur];
    cur ^= 1;
  }
  TS_TRY(scale_inverse_fp64(p, sigma, buf[cur ^ 1], s));
  for (int k = 0; k < p->d; ++k) {
    double* dst = (k == p->d - 1) ? u : buf[cur];
    TS_TRY(rot_pass_fp64(src, dst, p->St[k], N / p->n[k], p->n[k], 1, s));
    src = dst;
    cur ^= 1;
  }
  return TS_OK;
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" ts_status ts_apply_inverse_noalloc(const ts_plan* plan, double sigma, const double* b, double* u,
                                              ts_precision prec, void* stream) {
  clear_error();
  TS_REQUIRE(plan, "plan is NULL");
  TS_REQUIRE(b && u, "b and u must be non-NULL");
  int prev = -1;
  TS_CHECK_CUDA(cudaGetDevice(&prev));
  if (prev != plan->device) TS_CHECK_CUDA(cudaSetDevice(plan->device));
  struct Restore {
    int dev;
    ~Restore() {
      if (dev >= 0) cudaSetDevice(dev);
    }
  } restore{prev != plan->device ? prev : -1};
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = plan->N;
  size_t per_buffer = 0;
  if (prec == TS_FP64) {
    per_buffer = sizeof(double) * (size_t)N;
  } else {
    const int np = bf16_planes(prec);
    if (np == 0) {
      set_error("ts_apply_inverse_noalloc supports TS_FP64, TS_BF16X3 and TS_BF16X6 (got %d)", (int)prec);
      return TS_ERR_UNSUPPORTED;
    }
    if (!(plan->precision_mask & (1u << prec))) {
      set_error("precision %d was not requested in the plan's precision_mask", (int)prec);
      return TS_ERR_UNSUPPORTED;
    }
    per_buffer = sizeof(__nv_bfloat16) * (size_t)np * (size_t)mixed_plane_elems(plan);
  }
  per_buffer = (per_buffer + 255) & ~size_t(255);
  if (2 * per_buffer > NOALLOC_SCRATCH_BYTES) {
    set_error("ts_apply_inverse_noalloc: N = %lld needs %zu bytes of scratch, above the fixed %zu bytes "
              "(at most %lld DoF for TS_FP64, %lld for TS_BF16X3, %lld for TS_BF16X6)",
              N, 2 * per_buffer, NOALLOC_SCRATCH_BYTES, (long long)(NOALLOC_SCRATCH_BYTES / 16),
              (long long)(NOALLOC_SCRATCH_BYTES / 8), (long long)(NOALLOC_SCRATCH_BYTES / 12));
    return TS_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  TS_TRY(scratch_address(&base));
  unsigned char* w0 = static_cast<unsigned char*>(base);
  unsigned char* w1 = w0 + per_buffer;
  if (prec == TS_FP64) return fp64_inverse_buffers(plan, sigma, b, u, (double*)w0, (double*)w1, s);
  return mixed_inverse_buffers(plan, prec, sigma, b, u, (__nv_bfloat16*)w0, (__nv_bfloat16*)w1, s);
}
