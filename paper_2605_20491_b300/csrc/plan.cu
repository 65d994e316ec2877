// Plan creation: step 1 of Sec. 2.1 (eq. eigen_decomp).
//
// For the Q^1 discretisation the mass matrix is M_k = h_k I, so
//     H_k = M_k^{-1} Stiff_k + F_k = h_k^{-2} tridiag(-1, 2, -1) + diag f_k(x_{k,i})
// is symmetric and T_k = S_k is orthogonal (T_k^{-1} = S_k^T).  For Q^k, k >= 2, M_k is the
// diagonal GLL mass and H_k is similar to the symmetric M^{-1/2} Stiff M^{-1/2} + F_k =
// Q Lambda Q^T, so T_k = M^{-1/2} Q and T_k^{-1} = Q^T M^{1/2}; the diagonal factors are
// folded into the contraction operands, so every apply kernel runs unchanged.  Each
// symmetric matrix is eigendecomposed in FP64 (eigenvalues ascending, eigenvectors as
// columns): the tridiagonal Q^1 operator up to TRIDIAG_HOST_MAX nodes on the host by
// implicit QR (no device synchronisation, so plan builders overlap the GPU work of others),
// every other one on the GPU (cuSOLVER syevd).  The tables stay resident on the device for
// every later apply, in the stream-ordered table pool.
//
// Axis tables are cached process-wide by (device, n, L, f): plans whose axes coincide
// -- within one plan (isotropic grids) or across plans (a server's stream of requests on
// a few distinct 1D operators) -- share one decomposition.  The cache keeps the most
// recently built tables alive even when no plan holds them.
#include <cusolverDn.h>

#include <cmath>
#include <cstring>
#include <deque>
#include <map>

#include "common.cuh"
#include "mixed.cuh"
#include "sem_axis.cuh"
#include "small_n.cuh"

namespace ts {

AxisTables::~AxisTables() {
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  table_free(block, device);
  for (int q = 0; q < NPREC; ++q) {
    table_free(Bf[q], device);
    table_free(Bb[q], device);
  }
  table_free(Sf32, device);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
}

namespace {

// One cuSOLVER handle and workspace per host thread, grown on demand.
struct Solver {
  int device = -1;
  cusolverDnHandle_t h = nullptr;
  double *dA = nullptr, *dW = nullptr, *work = nullptr;
  int* info = nullptr;
  int cap_n = 0, cap_work = 0;
  void release() {
    if (h) cusolverDnDestroy(h);
    cudaFree(dA);
    cudaFree(dW);
    cudaFree(work);
    cudaFree(info);
    *this = Solver();
  }
};
thread_local Solver t_solver;

ts_status eig_on_device(int n, const std::vector<double>& H, std::vector<double>& lam, std::vector<double>& Qcol,
                        cudaStream_t s) {
  Solver& sv = t_solver;
  int dev = 0;
  TS_CHECK_CUDA(cudaGetDevice(&dev));
  if (sv.h && sv.device != dev) sv.release();
  if (!sv.h) {
    if (cusolverDnCreate(&sv.h) != CUSOLVER_STATUS_SUCCESS) {
      set_error("cusolverDnCreate failed");
      return TS_ERR_CUDA;
    }
    sv.device = dev;
    TS_CHECK_CUDA(cudaMalloc(&sv.info, sizeof(int)));
  }
  cusolverDnSetStream(sv.h, s);
  if (n > sv.cap_n) {
    cudaFree(sv.dA);
    cudaFree(sv.dW);
    sv.dA = sv.dW = nullptr;
    TS_CHECK_CUDA(cudaMalloc(&sv.dA, sizeof(double) * n * n));
    TS_CHECK_CUDA(cudaMalloc(&sv.dW, sizeof(double) * n));
    sv.cap_n = n;
  }
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(sv.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, sv.dA, n, sv.dW,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd_bufferSize failed");
    return TS_ERR_CUDA;
  }
  if (lwork > sv.cap_work) {
    cudaFree(sv.work);
    sv.work = nullptr;
    TS_CHECK_CUDA(cudaMalloc(&sv.work, sizeof(double) * (lwork > 0 ? lwork : 1)));
    sv.cap_work = lwork;
  }
  TS_CHECK_CUDA(cudaMemcpyAsync(sv.dA, H.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
  if (cusolverDnDsyevd(sv.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, sv.dA, n, sv.dW, sv.work, lwork,
                       sv.info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd failed");
    return TS_ERR_CUDA;
  }
  lam.resize(n);
  Qcol.resize((size_t)n * n);
  int hinfo = 0;
  TS_CHECK_CUDA(cudaMemcpyAsync(lam.data(), sv.dW, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(Qcol.data(), sv.dA, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(&hinfo, sv.info, sizeof(int), cudaMemcpyDeviceToHost, s));
  TS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (hinfo != 0) {
    set_error("syevd returned info = %d", hinfo);
    return TS_ERR_CUDA;
  }
  return TS_OK;
}

struct AxisKey {
  int device, n;
  double L;
  std::vector<double> f;
  int order, frame;
  bool operator<(const AxisKey& o) const {
    if (device != o.device) return device < o.device;
    if (n != o.n) return n < o.n;
    if (order != o.order) return order < o.order;
    if (frame != o.frame) return frame < o.frame;
    const int c = std::memcmp(&L, &o.L, sizeof(double));
    if (c != 0) return c < 0;
    return std::memcmp(f.data(), o.f.data(), sizeof(double) * f.size()) < 0;
  }
};

std::mutex g_axis_mu;
std::map<AxisKey, std::weak_ptr<AxisTables>> g_axis_map;
std::deque<std::shared_ptr<AxisTables>> g_axis_keep;
constexpr size_t AXIS_KEEP = 128;
long long g_axis_hits = 0, g_axis_builds = 0;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

ts_status build_axis(const AxisKey& key, cudaStream_t s, std::shared_ptr<AxisTables>* out) {
  auto t = std::make_shared<AxisTables>();
  const int n = key.n;
  t->device = key.device;
  t->n = n;
  t->L = key.L;
  t->f = key.f;
  t->order = key.order;
  t->frame = key.frame;
  const bool hermite = key.order == ORDER_HERMITE;
  const bool sem = key.order >= 2 || hermite;  // a diagonal M other than h I, and a band table
  std::vector<double> H((size_t)n * n, 0.0);
  SemAxis ax;
  HermiteAxis hx;
  std::vector<double> rh(n, 1.0), rhi(n, 1.0);  // M^{1/2}, M^{-1/2} (Q^k, Hermite)
  if (hermite) {
    // -D^2 + F = W^{-1/2} (-B^2 + F) W^{1/2} (W: the Gauss weights of Hermite functions)
    TS_TRY(hermite_axis_build(n, &hx));
    for (int i = 0; i < n; ++i) {
      rh[i] = std::exp(0.5 * hx.log_w[i]);
      rhi[i] = std::exp(-0.5 * hx.log_w[i]);
      for (int j = 0; j < n; ++j) H[(size_t)i * n + j] = hx.hs0[(size_t)i * n + j] + (i == j ? key.f[i] : 0.0);
    }
  } else if (!sem) {
    const double h = 2.0 * key.L / (n + 1);
    const double ih2 = 1.0 / (h * h);
    for (int i = 0; i < n; ++i) {
      H[(size_t)i * n + i] = 2.0 * ih2 + key.f[i];
      if (i > 0) H[(size_t)i * n + i - 1] = -ih2;
      if (i + 1 < n) H[(size_t)i * n + i + 1] = -ih2;
    }
  } else {
    TS_TRY(sem_axis_build(n, key.L, key.order, &ax));
    for (int i = 0; i < n; ++i) {
      rh[i] = std::sqrt(ax.m[i]);
      rhi[i] = 1.0 / rh[i];
    }
    // M^{-1/2} Stiff M^{-1/2} + diag f; the assembled Stiff is symmetric, so is this
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        H[(size_t)i * n + j] = rhi[i] * ax.stiff[(size_t)i * n + j] * rhi[j] + (i == j ? key.f[i] : 0.0);
  }
  std::vector<double> Qcol;
  if (!sem && n <= TRIDIAG_HOST_MAX) {  // Q^1: H is tridiagonal already
    std::vector<double> dg(n), od(n > 1 ? n - 1 : 1, 0.0);
    for (int i = 0; i < n; ++i) dg[i] = H[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) od[i] = H[(size_t)i * n + i + 1];
    t->lam_host.resize(n);
    Qcol.resize((size_t)n * n);
    if (!tridiag_eig_host(n, dg.data(), od.data(), t->lam_host.data(), Qcol.data()))
      TS_TRY(eig_on_device(n, H, t->lam_host, Qcol, s));
  } else {
    TS_TRY(eig_on_device(n, H, t->lam_host, Qcol, s));
  }
  // Qcol is column-major: Qcol[i + n j] = Q[i][j].  Forward operand S[i][j] = M^{1/2}_i Q[i][j],
  // backward operand St[j][i] = Q[i][j] M^{-1/2}_i; in frame 1 (and for Q^1) Q and Q^T.
  const bool fold = sem && key.frame == 0;
  std::vector<double> Sh((size_t)n * n), Sth((size_t)n * n);
  t->S_host.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double q = Qcol[(size_t)i + (size_t)n * j];
      Sh[(size_t)i * n + j] = fold ? rh[i] * q : q;
      Sth[(size_t)j * n + i] = fold ? rhi[i] * q : q;
      t->S_host[(size_t)i * n + j] = key.frame == 0 ? rhi[i] * q : q;
    }
  // the band of K = M^{-1} Stiff (frame 0) or M^{-1/2} Stiff M^{-1/2} (frame 1); Hermite: K is
  // dense (half-width n - 1), -D^2 = W^{-1/2} (-B^2) W^{1/2} in frame 0 and -B^2 in frame 1
  const int hw = hermite ? n - 1 : key.order;
  const int bw = sem ? 2 * hw + 1 : 0;
  std::vector<double> band((size_t)n * bw, 0.0);
  for (int i = 0; i < n && sem; ++i)
    for (int o = 0; o < bw; ++o) {
      const int j = i + o - hw;
      if (j < 0 || j >= n) continue;
      if (hermite) {
        const double a = hx.hs0[(size_t)i * n + j];
        band[(size_t)i * bw + o] = key.frame == 0 ? std::exp(0.5 * (hx.log_w[j] - hx.log_w[i])) * a : a;
        continue;
      }
      const double a = ax.stiff[(size_t)i * n + j];
      band[(size_t)i * bw + o] = key.frame == 0 ? a / ax.m[i] : rhi[i] * a * rhi[j];
    }
  std::vector<float> lf(t->lam_host.begin(), t->lam_host.end());
  const size_t oS = 0, oSt = align256(oS + 8ull * n * n), oLam = align256(oSt + 8ull * n * n),
               oF = align256(oLam + 8ull * n), oLf = align256(oF + 8ull * n), oBand = align256(oLf + 4ull * n),
               oMh = align256(oBand + 8ull * n * bw), oMhi = align256(oMh + (sem ? 8ull * n : 0)),
               total = align256(oMhi + (sem ? 8ull * n : 0));
  TS_TRY(table_alloc(&t->block, total, s));
  t->bytes = (long long)total;
  char* b = (char*)t->block;
  t->S = (double*)(b + oS);
  t->St = (double*)(b + oSt);
  t->lam = (double*)(b + oLam);
  t->fdev = (double*)(b + oF);
  t->lamf = (float*)(b + oLf);
  TS_CHECK_CUDA(cudaMemcpyAsync(t->S, Sh.data(), 8ull * n * n, cudaMemcpyHostToDevice, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(t->St, Sth.data(), 8ull * n * n, cudaMemcpyHostToDevice, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(t->lam, t->lam_host.data(), 8ull * n, cudaMemcpyHostToDevice, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(t->fdev, key.f.data(), 8ull * n, cudaMemcpyHostToDevice, s));
  TS_CHECK_CUDA(cudaMemcpyAsync(t->lamf, lf.data(), 4ull * n, cudaMemcpyHostToDevice, s));
  if (sem) {
    t->band = (double*)(b + oBand);
    t->mh = (double*)(b + oMh);
    t->mhi = (double*)(b + oMhi);
    TS_CHECK_CUDA(cudaMemcpyAsync(t->band, band.data(), 8ull * n * bw, cudaMemcpyHostToDevice, s));
    TS_CHECK_CUDA(cudaMemcpyAsync(t->mh, rh.data(), 8ull * n, cudaMemcpyHostToDevice, s));
    TS_CHECK_CUDA(cudaMemcpyAsync(t->mhi, rhi.data(), 8ull * n, cudaMemcpyHostToDevice, s));
  }
  TS_CHECK_CUDA(cudaStreamSynchronize(s));  // host staging vectors go out of scope
  *out = t;
  return TS_OK;
}

ts_status get_axis(int device, int n, double L, const double* f, int order, int frame, cudaStream_t s,
                   std::shared_ptr<AxisTables>* out) {
  AxisKey key{device, n, L, std::vector<double>(f, f + n), order, frame};
  {
    std::lock_guard<std::mutex> lk(g_axis_mu);
    auto it = g_axis_map.find(key);
    if (it != g_axis_map.end()) {
      if (auto sp = it->second.lock()) {
        ++g_axis_hits;
        *out = sp;
        return TS_OK;
      }
    }
  }
  std::shared_ptr<AxisTables> built;
  TS_TRY(build_axis(key, s, &built));
  std::vector<std::shared_ptr<AxisTables>> evicted;  // destroyed after the lock is released
  std::lock_guard<std::mutex> lk(g_axis_mu);
  auto it = g_axis_map.find(key);
  if (it != g_axis_map.end()) {
    if (auto sp = it->second.lock()) {  // another thread built it meanwhile: use that one
      *out = sp;
      return TS_OK;
    }
  }
  ++g_axis_builds;
  g_axis_map[key] = built;
  g_axis_keep.push_back(built);
  while (g_axis_keep.size() > AXIS_KEEP) {
    evicted.push_back(std::move(g_axis_keep.front()));
    g_axis_keep.pop_front();
  }
  for (auto m = g_axis_map.begin(); m != g_axis_map.end();)  // drop dead entries
    m = m->second.expired() ? g_axis_map.erase(m) : std::next(m);
  *out = built;
  return TS_OK;
}

}  // namespace

void axis_cache_counters(long long* hits, long long* builds) {
  std::lock_guard<std::mutex> lk(g_axis_mu);
  if (hits) *hits = g_axis_hits;
  if (builds) *builds = g_axis_builds;
}

void plan_free(ts_plan* p) { delete p; }

namespace {
ts_status plan_create_frame(const ts_plan_desc* desc, unsigned mask, int frame, cudaStream_t s, ts_plan** out);
}

ts_status plan_create(const ts_plan_desc* desc, unsigned mask, cudaStream_t s, ts_plan** out) {
  TS_TRY(plan_create_frame(desc, mask, 0, s, out));
  if (banded_plan(*out)) {  // the symmetric frame used by PCG and inverse iteration
    const ts_status st = plan_create_frame(desc, mask, 1, s, &(*out)->sym);
    if (st != TS_OK) {
      plan_free(*out);
      *out = nullptr;
      return st;
    }
    (*out)->bytes += (*out)->sym->bytes;
  }
  return TS_OK;
}

namespace {
ts_status plan_create_frame(const ts_plan_desc* desc, unsigned mask, int frame, cudaStream_t s, ts_plan** out) {
  ts_plan* p = new ts_plan();
  ts_status st = TS_OK;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    st = TS_ERR_CUDA;
  }
  p->d = desc->d;
  p->N = 1;
  p->precision_mask = mask | 1u;
  p->order = desc->order >= 2 || desc->order == ORDER_HERMITE ? desc->order : 1;
  for (int k = 0; k < p->d; ++k) {
    p->n[k] = desc->n[k];
    p->L[k] = desc->L[k];
    p->N *= desc->n[k];
    if (desc->n[k] > p->nmax) p->nmax = desc->n[k];
  }
  for (int k = 0; k < p->d && st == TS_OK; ++k) {
    st = get_axis(p->device, p->n[k], p->L[k], desc->f[k], p->order, banded_plan(p) ? frame : 0, s, &p->axis[k]);
    if (st != TS_OK) break;
    AxisTables* t = p->axis[k].get();
    p->S[k] = t->S;
    p->St[k] = t->St;
    p->lam[k] = t->lam;
    p->lamf[k] = t->lamf;
    p->f[k] = t->fdev;
    p->band[k] = t->band;
    p->mh[k] = t->mh;
    p->mhi[k] = t->mhi;
  }
  for (int q = 1; q < NPREC && st == TS_OK; ++q) {
    if (!(p->precision_mask & (1u << q))) continue;
    st = q == TS_FP32 ? build_small_tables(p, s) : build_split_tables(p, (ts_precision)q, s);
  }
  for (int k = 0; k < p->d && st == TS_OK; ++k) {
    bool seen = false;
    for (int j = 0; j < k; ++j) seen |= p->axis[j].get() == p->axis[k].get();
    if (!seen) p->bytes += p->axis[k]->bytes;
  }
  if (st != TS_OK) {
    plan_free(p);
    *out = nullptr;
    return st;
  }
  *out = p;
  return TS_OK;
}
}  // namespace

}  // namespace ts

ts_plan::~ts_plan() { delete sym; }
