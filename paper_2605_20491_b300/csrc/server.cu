// Serving runtime: continuous batching of solve, propagation and PCG requests on one GPU.
//
// A scheduler thread owns the device work:
//   * admission: requests whose plan is built leave the queue, in submission order, while
//     fewer than max_inflight are on the GPU and their scratch footprint fits the
//     device-memory budget (requests that can never fit fail with TS_ERR_NO_MEMORY);
//     requests that arrive while others run are admitted as slots and memory free up;
//   * plans: planner threads (ts_server_config.planner_threads, 4 by default) build each
//     request's plan ahead of admission, overlapping the GPU work of earlier requests (for Q^1 axes
//     of up to 192 nodes no step of a build synchronises the device), from a plan cache
//     keyed by the grid and the sampled V1
//     (n_k, L_k, f_k compared bit for bit); the per-axis eigendecompositions underneath
//     are shared process-wide, so requests on a few distinct 1D operators rarely solve one;
//   * batching: the inverse / exp requests admitted in one scheduling round are captured
//     into ONE CUDA graph and launched.  Split-precision requests run as one batched apply
//     (mixed_apply_batch: one input-split launch and, for each of the 2d passes, one
//     work-list tensor-core launch over the tiles of all of them); FP64 requests run on
//     their own forked streams, so their kernels overlap; the graph's completion event completes
//     every request of the batch;
//   * PCG requests read one scalar back per iteration, so they cannot live in a graph: each
//     runs on a pooled host thread with its own stream, overlapping with everything else.
// Results do not depend on what else runs: every kernel's work split and every reduction
// order is fixed by the problem size alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "mixed.cuh"
#include "solvers.cuh"

ts_status ts_plan_create(const ts_plan_desc*, unsigned, void*, ts_plan**);
ts_status ts_plan_destroy(ts_plan*);

namespace ts {
namespace {

using Clock = std::chrono::steady_clock;

struct PlanKey {
  int d;
  int order = 1;          // the k of Q^k
  std::vector<int> n;
  std::vector<double> L;
  std::vector<double> f;  // all axes' samples concatenated
  bool operator<(const PlanKey& o) const {
    if (d != o.d) return d < o.d;
    if (order != o.order) return order < o.order;
    if (n != o.n) return n < o.n;
    if (L != o.L) return L < o.L;
    return std::lexicographical_compare(f.begin(), f.end(), o.f.begin(), o.f.end(), [](double a, double b) {
      uint64_t x, y;
      std::memcpy(&x, &a, 8);
      std::memcpy(&y, &b, 8);
      return x < y;
    });
  }
};

using PlanPtr = std::shared_ptr<ts_plan>;

struct Job {
  long long ticket = 0;
  ts_request req{};
  PlanKey key;
  std::vector<std::vector<double>> f;  // copies of the V1 samples
  PlanPtr plan_ref;                     // keeps the plan alive while the job runs
  ts_plan* plan = nullptr;
  bool plan_ready = false;
  ts_status plan_status = TS_OK;
  size_t footprint = 0;
  Clock::time_point t_submit, t_done;
  int stream_slot = -1;
  ts_status status = TS_OK;
  int iterations = 0;
  bool done = false;
  char msg[256] = "";
};

// Np: elements of one bf16 plane (the grid with each pass's contracted axis padded to a
// multiple of 8, maximised over the passes).
size_t footprint_of(const ts_request& r, long long N, long long Np) {
  const int np = bf16_planes(r.prec);
  size_t apply_scratch;
  if (r.kind == TS_REQ_EXP) {
    apply_scratch = np ? 2 * (size_t)2 * np * Np * 2 : 2 * (size_t)2 * N * 8;
    if (np == 0 && r.dtype == TS_C64) apply_scratch += (size_t)2 * N * 8;
  } else {
    apply_scratch = np ? 2 * (size_t)np * Np * 2 : 2 * (size_t)N * 8;
  }
  if (r.kind == TS_REQ_PCG) apply_scratch += (size_t)4 * N * 8 + 16 * 1024;
  return apply_scratch + (1 << 20);
}

}  // namespace
}  // namespace ts

struct ts_server {
  ts_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::list<std::shared_ptr<ts::Job>> pending;  // submission order
  // PCG requests: a queue served by max_inflight persistent host threads (each keeps its
  // pinned residual mailbox and events for its lifetime)
  std::deque<std::shared_ptr<ts::Job>> pcg_queue;
  std::condition_variable cv_pcg;
  std::vector<std::thread> pcg_workers;
  bool pcg_stop = false;
  std::map<long long, std::shared_ptr<ts::Job>> jobs;
  long long next_ticket = 1;
  size_t mem_used = 0, mem_peak = 0;
  int inflight = 0;
  bool stop = false;
  std::thread worker;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  cudaStream_t capture_stream = nullptr;
  std::map<ts::PlanKey, ts::PlanPtr> plans;
  std::deque<ts::PlanKey> plan_lru;
  std::mutex plan_mu;
  std::condition_variable cv_plan;
  std::deque<std::shared_ptr<ts::Job>> to_plan;
  std::vector<std::thread> planners;
  std::vector<cudaStream_t> planner_streams;
  long long plan_hits = 0, plan_misses = 0, batches = 0, graph_requests = 0;
  std::vector<double> latencies_ms;
  double dof_done = 0.0;
  ts::Clock::time_point t_first{}, t_last{};
  bool have_first = false;
  struct Batch {
    std::vector<std::shared_ptr<ts::Job>> jobs;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Batch> batches_inflight;
};

namespace ts {
namespace {

// Plan of a job from the server's cache, built on a miss (called by planner threads).
ts_status get_plan(ts_server* sv, Job& j, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lk(sv->plan_mu);
    auto it = sv->plans.find(j.key);
    if (it != sv->plans.end()) {
      ++sv->plan_hits;
      j.plan_ref = it->second;
      j.plan = j.plan_ref.get();
      return TS_OK;
    }
  }
  std::vector<const double*> fp(j.key.d);
  for (int k = 0; k < j.key.d; ++k) fp[k] = j.f[k].data();
  ts_plan_desc desc = j.req.grid;
  desc.d = j.key.d;
  desc.f = fp.data();
  desc.n = j.key.n.data();
  desc.L = j.key.L.data();
  unsigned mask = (1u << TS_BF16X3) | (1u << TS_BF16X6);
  bool small = true;
  for (int k = 0; k < j.key.d; ++k) small &= j.key.n[k] == 8 || j.key.n[k] == 16 || j.key.n[k] == 24 || j.key.n[k] == 32;
  if (small) mask |= 1u << TS_FP32;
  ts_plan* p = nullptr;
  TS_TRY(ts_plan_create(&desc, mask, s, &p));
  PlanPtr pp(p, [](ts_plan* q) { ts_plan_destroy(q); });
  std::lock_guard<std::mutex> lk(sv->plan_mu);
  auto it = sv->plans.find(j.key);
  if (it != sv->plans.end()) {
    pp = it->second;  // built concurrently by another planner
  } else {
    ++sv->plan_misses;
    sv->plans[j.key] = pp;
    sv->plan_lru.push_back(j.key);
    while ((int)sv->plan_lru.size() > sv->cfg.plan_cache_entries) {  // running jobs keep their own reference
      sv->plans.erase(sv->plan_lru.front());
      sv->plan_lru.pop_front();
    }
  }
  j.plan_ref = pp;
  j.plan = pp.get();
  return TS_OK;
}

void planner_loop(ts_server* sv, int idx) {
  cudaSetDevice(sv->device);
  while (true) {
    std::shared_ptr<Job> jp;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_plan.wait(lk, [&] { return sv->stop || !sv->to_plan.empty(); });
      if (sv->to_plan.empty()) return;
      jp = sv->to_plan.front();
      sv->to_plan.pop_front();
    }
    ts_status st = get_plan(sv, *jp, sv->planner_streams[idx]);
    char msg[256] = "";
    if (st != TS_OK) snprintf(msg, sizeof(msg), "%s", ts_last_error());
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      jp->plan_status = st;
      if (st != TS_OK) snprintf(jp->msg, sizeof(jp->msg), "%s", msg);
      jp->plan_ready = true;
    }
    sv->cv_work.notify_all();
  }
}

ts_status enqueue_async(const Job& j, cudaStream_t s) {
  const ts_request& r = j.req;
  if (r.kind == TS_REQ_INVERSE)
    return apply_inverse_impl(j.plan, r.sigma, (const double*)r.in, (double*)r.out, r.prec, s);
  return apply_exp_impl(j.plan, r.tau, r.in, r.out, r.dtype, r.prec, s);
}

void finish(ts_server* sv, Job& j, ts_status st) {
  j.status = st;
  j.t_done = Clock::now();
  j.done = true;
  const double ms = std::chrono::duration<double, std::milli>(j.t_done - j.t_submit).count();
  sv->latencies_ms.push_back(ms);
  sv->dof_done += (double)(j.plan ? j.plan->N : 0);
  j.plan_ref.reset();  // the cache may drop the plan now
  if (!sv->have_first || j.t_submit < sv->t_first) sv->t_first = j.t_submit;
  sv->have_first = true;
  if (j.t_done > sv->t_last) sv->t_last = j.t_done;
  sv->mem_used -= j.footprint;
  --sv->inflight;
  if (j.stream_slot >= 0) sv->stream_busy[j.stream_slot] = false;
}

void run_pcg(ts_server* sv, std::shared_ptr<Job> jp) {
  Job& j = *jp;
  cudaSetDevice(sv->device);
  const ts_request& r = j.req;
  int it = 0;
  ts_status st = pcg_solve(j.plan, r.sigma, r.sigma, r.V2, (const double*)r.in, (double*)r.out, r.tol, r.maxit,
                          r.prec, &it, nullptr, sv->streams[j.stream_slot]);
  if (st != TS_OK) snprintf(j.msg, sizeof(j.msg), "%s", ts_last_error());
  std::lock_guard<std::mutex> lk(sv->mu);
  j.iterations = it;
  finish(sv, j, st);
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

void pcg_worker_loop(ts_server* sv) {
  cudaSetDevice(sv->device);
  while (true) {
    std::shared_ptr<Job> jp;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_pcg.wait(lk, [&] { return sv->pcg_stop || !sv->pcg_queue.empty(); });
      if (sv->pcg_queue.empty()) return;
      jp = sv->pcg_queue.front();
      sv->pcg_queue.pop_front();
    }
    run_pcg(sv, jp);
  }
}

void worker_loop(ts_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // 1. completions of launched graphs
    for (size_t b = 0; b < sv->batches_inflight.size();) {
      auto& bt = sv->batches_inflight[b];
      if (cudaEventQuery(bt.done) == cudaSuccess) {
        for (auto& jp : bt.jobs) finish(sv, *jp, TS_OK);
        cudaGraphExecDestroy(bt.exec);
        cudaGraphDestroy(bt.graph);
        cudaEventDestroy(bt.done);
        sv->batches_inflight.erase(sv->batches_inflight.begin() + b);
        sv->cv_done.notify_all();
      } else {
        ++b;
      }
    }
    if (sv->stop && sv->pending.empty() && sv->inflight == 0) break;
    // 2. admission, in submission order among the requests whose plan is built: a request
    //    still waiting for its plan does not hold back later ones.  A built request that does
    //    not fit the memory left stops the scan, so that smaller ones cannot starve it.
    std::vector<std::shared_ptr<Job>> batch, pcg;
    for (auto it = sv->pending.begin(); it != sv->pending.end() && sv->inflight < sv->cfg.max_inflight &&
                                        (int)batch.size() < sv->cfg.max_batch;) {
      auto jp = *it;
      if (!jp->plan_ready) {
        ++it;
        continue;
      }
      if (jp->footprint > (size_t)sv->cfg.memory_budget_bytes) {
        it = sv->pending.erase(it);
        snprintf(jp->msg, sizeof(jp->msg), "request needs %zu bytes of scratch, above the budget %lld",
                 jp->footprint, sv->cfg.memory_budget_bytes);
        ++sv->inflight;
        sv->mem_used += jp->footprint;
        finish(sv, *jp, TS_ERR_NO_MEMORY);
        sv->cv_done.notify_all();
        continue;
      }
      if (sv->mem_used + jp->footprint > (size_t)sv->cfg.memory_budget_bytes) break;
      int slot = -1;
      for (int q = 0; q < (int)sv->streams.size(); ++q)
        if (!sv->stream_busy[q]) {
          slot = q;
          break;
        }
      if (slot < 0) break;
      it = sv->pending.erase(it);
      ts_status st = jp->plan_status;
      if (st != TS_OK) {
        ++sv->inflight;
        sv->mem_used += jp->footprint;
        finish(sv, *jp, st);
        sv->cv_done.notify_all();
        continue;
      }
      sv->stream_busy[slot] = true;
      jp->stream_slot = slot;
      sv->mem_used += jp->footprint;
      sv->mem_peak = std::max(sv->mem_peak, sv->mem_used);
      ++sv->inflight;
      (jp->req.kind == TS_REQ_PCG ? pcg : batch).push_back(jp);
    }
    // 3. launch: PCG on the pooled host threads, the rest as one captured graph
    for (auto& jp : pcg) sv->pcg_queue.push_back(jp);
    if (!pcg.empty()) sv->cv_pcg.notify_all();
    if (!batch.empty()) {
      ts_server::Batch bt;
      bt.jobs = batch;
      cudaStream_t cs = sv->capture_stream;
      ts_status st = TS_OK;
      cudaEvent_t fork = nullptr;
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      std::vector<cudaEvent_t> joins(batch.size(), nullptr);
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = TS_ERR_CUDA;
      if (st == TS_OK) cudaEventRecord(fork, cs);
      // split-precision requests: every stage of all of them in one work-list launch
      // (mixed_apply_batch) on the capture stream; FP64 requests on their own forked streams
      std::vector<BatchApply> grouped;
      for (auto& jp : batch)
        if (bf16_planes(jp->req.prec) > 0) {
          const ts_request& r = jp->req;
          grouped.push_back(BatchApply{jp->plan, r.prec,
                                       r.kind == TS_REQ_INVERSE ? MixedOp::Inverse : MixedOp::Exp,
                                       r.kind == TS_REQ_INVERSE ? r.sigma : r.tau, r.in, r.out,
                                       r.kind == TS_REQ_INVERSE ? TS_R64 : r.dtype});
        }
      if (st == TS_OK && !grouped.empty()) {
        st = mixed_apply_batch(grouped.data(), (int)grouped.size(), cs);
        if (st != TS_OK)
          for (auto& jp : batch)
            if (bf16_planes(jp->req.prec) > 0) snprintf(jp->msg, sizeof(jp->msg), "%s", ts_last_error());
      }
      for (size_t q = 0; q < batch.size() && st == TS_OK; ++q) {
        if (bf16_planes(batch[q]->req.prec) > 0) continue;
        cudaStream_t s = sv->streams[batch[q]->stream_slot];
        cudaStreamWaitEvent(s, fork, 0);
        st = enqueue_async(*batch[q], s);
        if (st != TS_OK) snprintf(batch[q]->msg, sizeof(batch[q]->msg), "%s", ts_last_error());
        cudaEventCreateWithFlags(&joins[q], cudaEventDisableTiming);
        cudaEventRecord(joins[q], s);
        cudaStreamWaitEvent(cs, joins[q], 0);
      }
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cs, &g);
      if (st == TS_OK && ce != cudaSuccess) st = TS_ERR_CUDA;
      if (st == TS_OK && cudaGraphInstantiate(&bt.exec, g, 0) != cudaSuccess) st = TS_ERR_CUDA;
      bt.graph = g;
      cudaEventDestroy(fork);
      for (auto e : joins)
        if (e) cudaEventDestroy(e);
      if (st == TS_OK) {
        cudaEventCreateWithFlags(&bt.done, cudaEventDisableTiming);
        cudaGraphLaunch(bt.exec, cs);
        cudaEventRecord(bt.done, cs);
        ++sv->batches;
        sv->graph_requests += (long long)batch.size();
        sv->batches_inflight.push_back(bt);
      } else {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        for (auto& jp : batch) {
          if (!jp->msg[0]) snprintf(jp->msg, sizeof(jp->msg), "batch capture failed");
          finish(sv, *jp, st);
        }
        sv->cv_done.notify_all();
      }
    }
    // 4. wait for new work or poll the GPU
    if (sv->batches_inflight.empty() && (sv->pending.empty() || sv->inflight >= sv->cfg.max_inflight))
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    else if (batch.empty() && pcg.empty()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
  lk.unlock();
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" {

namespace {

// Streams, kernels and threads of a new server; the threads start only after every CUDA
// call has succeeded, so a failure leaves only streams for the caller to release.
ts_status server_init(ts_server* sv) {
  TS_REQUIRE(sv->cfg.max_inflight <= TS_SERVER_MAX_INFLIGHT, "max_inflight %d is above %d", sv->cfg.max_inflight,
             TS_SERVER_MAX_INFLIGHT);
  if (sv->cfg.max_inflight <= 0) sv->cfg.max_inflight = 8;
  if (sv->cfg.max_batch <= 0) sv->cfg.max_batch = sv->cfg.max_inflight;
  if (sv->cfg.plan_cache_entries <= 0) sv->cfg.plan_cache_entries = 1024;
  TS_CHECK_CUDA(cudaGetDevice(&sv->device));
  if (sv->cfg.memory_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    TS_CHECK_CUDA(cudaMemGetInfo(&fr, &tot));
    sv->cfg.memory_budget_bytes = (long long)(fr / 2);
  }
  sv->streams.resize(sv->cfg.max_inflight);
  sv->stream_busy.assign(sv->cfg.max_inflight, false);
  for (auto& s : sv->streams) TS_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  TS_CHECK_CUDA(cudaStreamCreateWithFlags(&sv->capture_stream, cudaStreamNonBlocking));
  TS_TRY(tc_prepare_kernels());
  scratch_pool_prepare();  // its attributes cannot be set inside the rounds' graph captures
  // Planners build plans on host threads (Q^1 eigendecompositions on the host, table
  // uploads and splits on their own streams); their streams take the highest priority, so
  // the few small kernels of a build are scheduled ahead of queued batch work.
  const int nplanners = sv->cfg.planner_threads > 0 ? (sv->cfg.planner_threads > 64 ? 64 : sv->cfg.planner_threads) : 4;
  int prio_least = 0, prio_greatest = 0;
  TS_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
  sv->planner_streams.resize(nplanners);
  for (auto& s : sv->planner_streams)
    TS_CHECK_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_greatest));
  for (int i = 0; i < nplanners; ++i) sv->planners.emplace_back(planner_loop, sv, i);
  for (int i = 0; i < sv->cfg.max_inflight; ++i) sv->pcg_workers.emplace_back(pcg_worker_loop, sv);
  sv->worker = std::thread(worker_loop, sv);
  return TS_OK;
}

}  // namespace

ts_status ts_server_create(const ts_server_config* cfg, ts_server** out) {
  clear_error();
  TS_REQUIRE(out, "out is NULL");
  *out = nullptr;
  ts_server* sv = new ts_server();
  if (cfg) sv->cfg = *cfg;
  const ts_status st = server_init(sv);
  if (st != TS_OK) {
    for (auto s : sv->streams)
      if (s) cudaStreamDestroy(s);
    for (auto s : sv->planner_streams)
      if (s) cudaStreamDestroy(s);
    if (sv->capture_stream) cudaStreamDestroy(sv->capture_stream);
    delete sv;
    return st;
  }
  *out = sv;
  return TS_OK;
}

ts_status ts_server_submit(ts_server* sv, const ts_request* r, long long* ticket) {
  clear_error();
  TS_REQUIRE(sv && r && ticket, "NULL argument");
  TS_REQUIRE(r->kind >= TS_REQ_INVERSE && r->kind <= TS_REQ_PCG, "unknown request kind %d", r->kind);
  TS_REQUIRE(r->grid.d >= 1 && r->grid.d <= TS_MAX_DIM && r->grid.n && r->grid.L && r->grid.f, "bad grid");
  TS_REQUIRE(r->in && r->out, "in and out must be non-NULL");
  if (r->kind == TS_REQ_EXP)
    TS_REQUIRE(r->dtype == TS_C128 || r->dtype == TS_C64, "exp requests need TS_C128 or TS_C64");
  else
    TS_REQUIRE(r->dtype == TS_R64, "inverse and PCG requests need TS_R64");
  TS_REQUIRE((int)r->prec >= 0 && (int)r->prec < NPREC, "bad precision");
  if (r->kind == TS_REQ_PCG) TS_REQUIRE(r->tol > 0 && r->maxit > 0 && r->in != r->out, "bad PCG parameters");
  auto jp = std::make_shared<Job>();
  jp->req = *r;
  jp->key.d = r->grid.d;
  TS_REQUIRE(r->grid.order >= -1 && r->grid.order <= 32, "bad order %d", r->grid.order);
  jp->key.order = r->grid.order >= 2 || r->grid.order == -1 ? r->grid.order : 1;
  long long N = 1;
  for (int k = 0; k < r->grid.d; ++k) {
    TS_REQUIRE(r->grid.n[k] >= 1 && r->grid.n[k] <= 4096 && r->grid.L[k] > 0 && r->grid.f[k], "bad axis %d", k);
    jp->key.n.push_back(r->grid.n[k]);
    jp->key.L.push_back(r->grid.L[k]);
    jp->f.emplace_back(r->grid.f[k], r->grid.f[k] + r->grid.n[k]);
    jp->key.f.insert(jp->key.f.end(), r->grid.f[k], r->grid.f[k] + r->grid.n[k]);
    N *= r->grid.n[k];
  }
  jp->req.grid.n = nullptr;  // the job keeps its own copies
  jp->req.grid.L = nullptr;
  jp->req.grid.f = nullptr;
  long long Np = 0;
  for (int k = 0; k < r->grid.d; ++k) {
    const long long e = (N / r->grid.n[k]) * ((r->grid.n[k] + 7) & ~7);
    Np = e > Np ? e : Np;
  }
  jp->footprint = footprint_of(*r, N, Np);
  jp->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    TS_REQUIRE(!sv->stop, "server is shutting down");
    jp->ticket = sv->next_ticket++;
    sv->jobs[jp->ticket] = jp;
    sv->pending.push_back(jp);
    sv->to_plan.push_back(jp);
    *ticket = jp->ticket;
  }
  sv->cv_plan.notify_one();
  sv->cv_work.notify_all();
  return TS_OK;
}

ts_status ts_server_wait(ts_server* sv, long long ticket, ts_status* result, double* latency_ms, int* iterations) {
  clear_error();
  TS_REQUIRE(sv, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  TS_REQUIRE(it != sv->jobs.end(), "unknown ticket %lld", ticket);
  auto jp = it->second;
  sv->cv_done.wait(lk, [&] { return jp->done; });
  if (result) *result = jp->status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(jp->t_done - jp->t_submit).count();
  if (iterations) *iterations = jp->iterations;
  if (jp->status != TS_OK) set_error("%s", jp->msg);
  sv->jobs.erase(it);
  return TS_OK;
}

ts_status ts_server_drain(ts_server* sv) {
  clear_error();
  TS_REQUIRE(sv, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv_done.wait(lk, [&] { return sv->pending.empty() && sv->inflight == 0; });
  return TS_OK;
}

ts_status ts_server_stats(ts_server* sv, ts_serving_stats* st) {
  clear_error();
  TS_REQUIRE(sv && st, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> v = sv->latencies_ms;
  std::sort(v.begin(), v.end());
  std::memset(st, 0, sizeof(*st));
  st->completed = (long long)v.size();
  if (!v.empty()) {
    st->p50_ms = v[(size_t)(0.50 * (v.size() - 1))];
    st->p99_ms = v[(size_t)(0.99 * (v.size() - 1))];
    st->max_ms = v.back();
  }
  st->makespan_ms = sv->have_first ? std::chrono::duration<double, std::milli>(sv->t_last - sv->t_first).count() : 0;
  st->gdofs = st->makespan_ms > 0 ? sv->dof_done / (st->makespan_ms * 1e-3) / 1e9 : 0.0;
  st->plan_hits = sv->plan_hits;
  st->plan_misses = sv->plan_misses;
  st->batches = sv->batches;
  st->graph_requests = sv->graph_requests;
  st->peak_scratch_bytes = (long long)sv->mem_peak;
  return TS_OK;
}

ts_status ts_server_reset_stats(ts_server* sv) {
  clear_error();
  TS_REQUIRE(sv, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->latencies_ms.clear();
  sv->dof_done = 0;
  sv->have_first = false;
  sv->plan_hits = sv->plan_misses = sv->batches = sv->graph_requests = 0;
  sv->mem_peak = sv->mem_used;
  return TS_OK;
}

ts_status ts_server_destroy(ts_server* sv) {
  clear_error();
  if (!sv) return TS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  sv->cv_plan.notify_all();
  if (sv->worker.joinable()) sv->worker.join();  // returns once every request has finished
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->pcg_stop = true;
  }
  sv->cv_pcg.notify_all();
  for (auto& t : sv->pcg_workers) t.join();
  for (auto& t : sv->planners) t.join();
  sv->plans.clear();
  for (auto s : sv->streams) cudaStreamDestroy(s);
  for (auto s : sv->planner_streams) cudaStreamDestroy(s);
  if (sv->capture_stream) cudaStreamDestroy(sv->capture_stream);
  delete sv;
  return TS_OK;
}

}  // extern "C"
