// Autotuner of the split-precision tensor-core pass: for each distinct contracted extent
// n of a plan and the data kind (real / complex), time the candidate tile configurations
// (K chunk 64 or 32; N-tile cap 256, 128 or 64; single CTAs or CTA pairs sharing each MMA)
// on a whole apply with CUDA events, keep the fastest through tc_config_set, and remember
// it in a plain-text cache file so later processes skip the search.
// Cache line: "<complex> <n> <prec> <bk> <bn_cap> <cluster> <ms>", cluster 1 (single CTAs)
// or TS_TC_PAIR; lines with any other cluster value are ignored.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "mixed.cuh"

namespace ts {
namespace {

struct Entry {
  int cplx, n, prec, bk, bn, cluster;
  double ms;
};

std::vector<Entry> read_cache(const char* path) {
  std::vector<Entry> out;
  if (!path || !*path) return out;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ss(line);
    Entry e{};
    if (ss >> e.cplx >> e.n >> e.prec >> e.bk >> e.bn >> e.cluster >> e.ms &&
        (e.cluster == 1 || e.cluster == TS_TC_PAIR))
      out.push_back(e);
  }
  return out;
}

void append_cache(const char* path, const Entry& e) {
  if (!path || !*path) return;
  std::ofstream out(path, std::ios::app);
  out << e.cplx << " " << e.n << " " << e.prec << " " << e.bk << " " << e.bn << " " << e.cluster << " " << e.ms << "\n";
}

ts_status time_apply(const ts_plan* p, ts_precision prec, bool cplx, void* in, void* out, cudaStream_t s,
                     int reps, double* ms) {
  cudaEvent_t e0, e1;
  TS_CHECK_CUDA(cudaEventCreate(&e0));
  TS_CHECK_CUDA(cudaEventCreate(&e1));
  auto run = [&]() -> ts_status {
    if (cplx) return mixed_apply(p, prec, MixedOp::Exp, 0.01, in, out, TS_C128, s);
    return mixed_apply(p, prec, MixedOp::Inverse, 1.0, in, out, TS_R64, s);
  };
  ts_status st = run();  // warm-up
  if (st == TS_OK) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == TS_OK; ++r) st = run();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess && st == TS_OK) {
      set_error("autotune timing failed: %s", cudaGetErrorString(e));
      st = TS_ERR_CUDA;
    }
    *ms = t / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" ts_status ts_autotune(const ts_plan* plan, ts_dtype dtype, ts_precision prec, const char* cache_path,
                                 int* tuned, void* stream) {
  clear_error();
  TS_REQUIRE(plan, "plan is NULL");
  TS_REQUIRE(dtype == TS_R64 || dtype == TS_C128, "dtype must be TS_R64 (inverse) or TS_C128 (exp)");
  TS_REQUIRE(bf16_planes(prec) > 0, "autotuning applies to the split precisions");
  TS_REQUIRE(plan->precision_mask & (1u << prec), "precision %d is not in the plan's mask", (int)prec);
  int prev = -1;
  TS_CHECK_CUDA(cudaGetDevice(&prev));
  if (prev != plan->device) TS_CHECK_CUDA(cudaSetDevice(plan->device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool cplx = dtype == TS_C128;
  const int cval = cplx ? 1 : 0;
  std::vector<Entry> cache = read_cache(cache_path);
  int searched = 0;
  void* in = nullptr;
  void* out = nullptr;
  ts_status st = TS_OK;
  std::vector<int> done;
  for (int k = 0; k < plan->d && st == TS_OK; ++k) {
    const int n = plan->n[k];
    bool seen = false;
    for (int v : done) seen |= v == n;
    if (seen) continue;
    done.push_back(n);
    const Entry* hit = nullptr;
    for (const Entry& e : cache)
      if (e.cplx == cval && e.n == n && e.prec == (int)prec) hit = &e;
    if (hit) {
      st = tc_config_set(cval, n, hit->bk, hit->bn, hit->cluster);
      continue;
    }
    if (!in) {
      const size_t bytes = sizeof(double) * (size_t)plan->N * (cplx ? 2 : 1);
      st = scratch_alloc(&in, bytes, s);
      if (st == TS_OK) st = scratch_alloc(&out, bytes, s);
      if (st == TS_OK && cudaMemsetAsync(in, 0x3f, bytes, s) != cudaSuccess) {
        set_error("autotune: memset failed");
        st = TS_ERR_CUDA;
      }
      if (st != TS_OK) break;
    }
    Entry best{cval, n, (int)prec, 64, 256, 1, 1e30};
    const int bks[2] = {64, 32};
    const int bns[3] = {256, 128, 64};
    const int clusters[2] = {1, TS_TC_PAIR};
    for (int bk : bks)
      for (int bn : bns)
        for (int cl : clusters) {
          if (st != TS_OK) break;
          if (2 * (cplx ? 2 : 1) * bn > 512) continue;
          st = tc_config_set(cval, n, bk, bn, cl);
          double ms = 0.0;
          if (st == TS_OK) st = time_apply(plan, prec, cplx, in, out, s, 3, &ms);
          if (st == TS_OK && ms < best.ms) {
            best.bk = bk;
            best.bn = bn;
            best.cluster = cl;
            best.ms = ms;
          }
        }
    if (st == TS_OK) {
      st = tc_config_set(cval, n, best.bk, best.bn, best.cluster);
      append_cache(cache_path, best);
      ++searched;
    }
  }
  scratch_free(in, s);
  scratch_free(out, s);
  if (st == TS_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("autotune: %s", cudaGetErrorString(e));
      st = TS_ERR_CUDA;
    }
  }
  if (prev != plan->device) cudaSetDevice(prev);
  if (tuned) *tuned = searched;
  return st;
}
