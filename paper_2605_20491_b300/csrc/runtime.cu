// Process-wide runtime services: the kernel launch counter, live per-kernel timing with
// CUDA events (used by the benchmark to measure the contraction kernels inside its timed
// region without a profiler), and the device memory pool of the resident axis tables.
#include <atomic>
#include <map>
#include <mutex>

#include "common.cuh"

namespace ts {

namespace {

std::atomic<long long> g_launches{0};

struct Record {
  cudaEvent_t e0, e1;
  int kind;
  double flops, bytes;
};

std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

void prof_begin_launch(cudaStream_t s, void** token) {
  *token = nullptr;
  // launches being captured into a graph are not timed (their events would become nodes)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, s);
  *token = (void*)e;
}

void prof_end_launch(cudaStream_t s, void* token, int kind, double flops, double bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e1 = take_event();
  cudaEventRecord(e1, s);
  g_records.push_back({(cudaEvent_t)token, e1, kind, flops, bytes});
}

namespace {
struct TablePools {
  std::mutex mu;
  std::map<int, cudaMemPool_t> pool;
  std::map<int, cudaStream_t> release;  // an otherwise idle stream: frees complete at once
};
// Never destroyed: tables cached process-wide are released during static destruction.
TablePools& table_pools() {
  static TablePools* t = new TablePools;
  return *t;
}
}  // namespace

ts_status table_alloc(void** ptr, size_t bytes, cudaStream_t s) {
  *ptr = nullptr;
  int dev = 0;
  TS_CHECK_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool = nullptr;
  {
    TablePools& tp = table_pools();
    std::lock_guard<std::mutex> lk(tp.mu);
    auto it = tp.pool.find(dev);
    if (it == tp.pool.end()) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      TS_CHECK_CUDA(cudaMemPoolCreate(&pool, &props));
      uint64_t keep = UINT64_MAX;
      TS_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
      cudaStream_t rs = nullptr;
      TS_CHECK_CUDA(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
      tp.pool[dev] = pool;
      tp.release[dev] = rs;
    } else {
      pool = it->second;
    }
  }
  const cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes > 0 ? bytes : 1, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("table allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    *ptr = nullptr;
    return TS_ERR_NO_MEMORY;
  }
  return TS_OK;
}

void table_free(void* ptr, int device) {
  if (!ptr) return;
  cudaStream_t rs = nullptr;
  {
    TablePools& tp = table_pools();
    std::lock_guard<std::mutex> lk(tp.mu);
    auto it = tp.release.find(device);
    if (it != tp.release.end()) rs = it->second;
  }
  if (rs && cudaFreeAsync(ptr, rs) != cudaSuccess) cudaGetLastError();  // at exit the runtime may be gone
}

}  // namespace ts

using namespace ts;

extern "C" {

long long ts_launch_count(void) { return g_launches.load(); }

ts_status ts_profile_begin(void) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_records) {
    g_event_pool.push_back(r.e0);
    g_event_pool.push_back(r.e1);
  }
  g_records.clear();
  g_prof_on = true;
  return TS_OK;
}

ts_status ts_profile_end(int kind, long long* launches, double* total_ms, double* flops, double* bytes) {
  clear_error();
  g_prof_on = false;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  long long cnt = 0;
  double ms = 0.0, fl = 0.0, by = 0.0;
  for (auto& r : g_records) {
    if (r.kind != kind) continue;
    TS_CHECK_CUDA(cudaEventSynchronize(r.e1));
    float t = 0.f;
    TS_CHECK_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
    ++cnt;
    ms += t;
    fl += r.flops;
    by += r.bytes;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  if (flops) *flops = fl;
  if (bytes) *bytes = by;
  return TS_OK;
}

}  // extern "C"
