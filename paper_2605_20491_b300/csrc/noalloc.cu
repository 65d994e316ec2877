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
//
// Host code cannot use the array's name as a device address.  scratch_address() asks the
// runtime for it (cudaGetSymbolAddress, with the plan's device current) on the first call
// in each CUDA context of a device, and again whenever that device's context has been
// replaced (cudaDeviceReset, or the primary context released and created anew), because
// the module -- and with it the array -- may then be loaded at another address.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "mixed.cuh"

namespace ts {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

// The address found for a device, and the unique ID (cuCtxGetId) of the context it was
// found in.  IDs are never reused within a process, so an entry from a context that has
// since been destroyed can never match the current one.
struct ScratchSlot {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_addr_mu;
ScratchSlot g_slot[MAX_DEVICES];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// ID of the calling thread's current CUDA context; false if there is none or the driver
// cannot tell (the caller then looks the address up again).
bool current_context_id(unsigned long long* id) {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current device's current context.  Set-up:
// the first call in a context resolves it with cudaGetSymbolAddress (the device must be
// current) and checks the result; later calls in the same context reuse it.
ts_status scratch_address(void** out) {
  int dev = 0;
  TS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device ordinal %d out of range for the no-allocation scratch", dev);
    return TS_ERR_UNSUPPORTED;
  }
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  ScratchSlot& slot = g_slot[dev];
  if (have_id && slot.ptr && slot.ctx_id == id) {
    *out = slot.ptr;
    return TS_OK;
  }
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    slot = ScratchSlot{};
    set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
    return TS_ERR_CUDA;
  }
  // the lookup makes the context current if it was not; without an ID nothing is cached
  unsigned long long id_now = 0;
  if (current_context_id(&id_now)) {
    slot.ptr = ptr;
    slot.ctx_id = id_now;
  } else {
    slot = ScratchSlot{};
  }
  *out = ptr;
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
  // the same precision checks, with the same statuses, as ts_apply_inverse
  if ((int)prec < 0 || (int)prec >= NPREC || (int)prec == 3 || (int)prec == 4) {
    set_error("invalid precision %d", (int)prec);
    return TS_ERR_INVALID_ARG;
  }
  if (prec != TS_FP64 && !(plan->precision_mask & (1u << prec))) {
    set_error("precision %d was not requested in the plan's precision_mask", (int)prec);
    return TS_ERR_UNSUPPORTED;
  }
  const int np = bf16_planes(prec);
  if (prec != TS_FP64 && np == 0) {
    set_error("ts_apply_inverse_noalloc supports TS_FP64, TS_BF16X1, TS_BF16X3 and TS_BF16X6 (got %d)", (int)prec);
    return TS_ERR_UNSUPPORTED;
  }
  // bytes per buffer: N doubles, or the np bf16 planes of the widest pass (each pass's
  // contracted axis padded to a multiple of 8 elements)
  size_t per_buffer = prec == TS_FP64 ? sizeof(double) * (size_t)N
                                      : sizeof(__nv_bfloat16) * (size_t)np * (size_t)mixed_plane_elems(plan);
  per_buffer = (per_buffer + 255) & ~size_t(255);
  if (2 * per_buffer > NOALLOC_SCRATCH_BYTES) {
    const long long per_value = prec == TS_FP64 ? 16 : 4LL * np;
    set_error("ts_apply_inverse_noalloc: this plan (N = %lld) needs 2 x %zu bytes of scratch in precision %d, "
              "above the fixed %zu bytes; the limit is %lld DoF when every n_k is a multiple of 8 "
              "(rows of other lengths are padded, which lowers it)",
              N, per_buffer, (int)prec, NOALLOC_SCRATCH_BYTES, (long long)NOALLOC_SCRATCH_BYTES / per_value);
    return TS_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  TS_TRY(scratch_address(&base));
  unsigned char* w0 = static_cast<unsigned char*>(base);
  unsigned char* w1 = w0 + per_buffer;
  if (prec == TS_FP64) return fp64_inverse_buffers(plan, sigma, b, u, (double*)w0, (double*)w1, s);
  return mixed_inverse_buffers(plan, prec, sigma, b, u, (__nv_bfloat16*)w0, (__nv_bfloat16*)w1, s);
}
