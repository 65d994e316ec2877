// Apply drivers: the direct inverse (steps 2-4 of Sec. 2.1) and the exact propagator
// (eq. exact_prop), composed of d rotating contraction passes forward, the pointwise
// eigenvalue scale or phase, and d passes backward.
#include <mutex>
#include <set>

#include "common.cuh"
#include "mixed.cuh"
#include "pointwise.cuh"
#include "small_n.cuh"

namespace ts {

namespace {
// The device's default pool serves the work buffers.  By default it hands freed memory
// back at every synchronisation, so a solver that synchronises between calls (one PCG
// solve per outer step of inverse iteration) maps its buffers afresh each time; keeping up
// to 4 GiB of freed buffers in the pool avoids that.  Setting a pool attribute is not
// allowed while a stream captures a graph: the first allocations of a process made under
// capture leave it for a later one (and ts_server_create sets it before any capture).
void keep_scratch_mapped() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (!done.insert(dev).second) return;
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = 4ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}
}  // namespace

void scratch_pool_prepare() { keep_scratch_mapped(); }

ts_status scratch_alloc(void** ptr, size_t bytes, cudaStream_t s) {
  *ptr = nullptr;
  if (bytes == 0) return TS_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // unknown: leave the pool alone this time
  }
  if (cs == cudaStreamCaptureStatusNone) keep_scratch_mapped();
  cudaError_t e = cudaMallocAsync(ptr, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    *ptr = nullptr;
    return TS_ERR_NO_MEMORY;
  }
  return TS_OK;
}

void scratch_free(void* ptr, cudaStream_t s) {
  if (ptr) cudaFreeAsync(ptr, s);
}

namespace {

// FP64 pipeline on real (ncomp 1) or interleaved complex (ncomp 2) FP64 data.
// in -> [d forward passes] -> pointwise(op) -> [d backward passes] -> out.
// in and out may alias: the first pass reads `in` into scratch and the last pass
// writes `out` from scratch.
ts_status fp64_pipeline(const ts_plan* p, const double* in, double* out, int ncomp, int op, double param,
                        cudaStream_t s) {
  const long long N = p->N;
  void* w0 = nullptr;
  void* w1 = nullptr;
  TS_TRY(scratch_alloc(&w0, sizeof(double) * N * ncomp, s));
  ts_status st = scratch_alloc(&w1, sizeof(double) * N * ncomp, s);
  if (st != TS_OK) {
    scratch_free(w0, s);
    return st;
  }
  double* buf[2] = {(double*)w0, (double*)w1};
  const double* src = in;
  int cur = 0;
  for (int k = 0; k < p->d && st == TS_OK; ++k) {   // forward: Y = X S_k
    st = rot_pass_fp64(src, buf[cur], p->S[k], N / p->n[k], p->n[k], ncomp, s);
    src = buf[cur];
    cur ^= 1;
  }
  double* coef = buf[cur ^ 1];
  if (st == TS_OK) {
    if (op == 0)
      st = scale_inverse_fp64(p, param, coef, s);
    else
      st = scale_exp_c128(p, param, coef, s);
  }
  for (int k = 0; k < p->d && st == TS_OK; ++k) {   // backward: Y = X S_k^T
    double* dst = (k == p->d - 1) ? out : buf[cur];
    st = rot_pass_fp64(src, dst, p->St[k], N / p->n[k], p->n[k], ncomp, s);
    src = dst;
    cur ^= 1;
  }
  scratch_free(w0, s);
  scratch_free(w1, s);
  return st;
}

}  // namespace

ts_status apply_inverse_impl(const ts_plan* p, double sigma, const double* b, double* u, ts_precision prec,
                             cudaStream_t s) {
  if (prec == TS_FP32) {
    set_error("TS_FP32 is available for complex64 propagation only");
    return TS_ERR_UNSUPPORTED;
  }
  if (prec == TS_FP64) return fp64_pipeline(p, b, u, 1, 0, sigma, s);
  return mixed_apply(p, prec, MixedOp::Inverse, sigma, b, u, TS_R64, s);
}

ts_status apply_exp_impl(const ts_plan* p, double tau, const void* in, void* out, ts_dtype dt, ts_precision prec,
                         cudaStream_t s) {
  if (prec == TS_FP32) {
    if (dt != TS_C64) {
      set_error("TS_FP32 propagation works on complex64 data");
      return TS_ERR_UNSUPPORTED;
    }
    return small_n_propagate(p, tau, (const float2*)in, (float2*)out, nullptr, tau, 1, s);
  }
  if (prec == TS_BF16X6 && dt == TS_C64 && small_tc_applicable(p))
    return small_n_propagate(p, tau, (const float2*)in, (float2*)out, nullptr, tau, 1, s, true);
  if (prec != TS_FP64) return mixed_apply(p, prec, MixedOp::Exp, tau, in, out, dt, s);
  if (dt == TS_C128) return fp64_pipeline(p, (const double*)in, (double*)out, 2, 1, tau, s);
  // complex64 data, FP64 arithmetic: widen, apply, narrow.
  void* w = nullptr;
  TS_TRY(scratch_alloc(&w, sizeof(double) * 2 * p->N, s));
  ts_status st = convert_c64_to_c128(p->N, (const float*)in, (double*)w, s);
  if (st == TS_OK) st = fp64_pipeline(p, (const double*)w, (double*)w, 2, 1, tau, s);
  if (st == TS_OK) st = convert_c128_to_c64(p->N, (const double*)w, (float*)out, s);
  scratch_free(w, s);
  return st;
}

}  // namespace ts
