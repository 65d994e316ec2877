// Plan creation: step 1 of Sec. 2.1 (eq. eigen_decomp).
//
// For the Q^1 discretisation the mass matrix is M_k = h_k I, so
//     H_k = M_k^{-1} Stiff_k + F_k = h_k^{-2} tridiag(-1, 2, -1) + diag f_k(x_{k,i})
// is symmetric and T_k = S_k is orthogonal (T_k^{-1} = S_k^T).  Each H_k is
// eigendecomposed in FP64 on the GPU (cuSOLVER syevd: eigenvalues ascending,
// eigenvectors as columns); the tables stay resident on the device for every later apply.
#include <cusolverDn.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "mixed.cuh"
#include "small_n.cuh"

namespace ts {

namespace {

ts_status eig_on_device(int n, const std::vector<double>& H, std::vector<double>& lam, std::vector<double>& Qcol,
                        cudaStream_t s) {
  cusolverDnHandle_t h = nullptr;
  if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnCreate failed");
    return TS_ERR_CUDA;
  }
  cusolverDnSetStream(h, s);
  double *dA = nullptr, *dW = nullptr, *work = nullptr;
  int* info = nullptr;
  ts_status st = TS_OK;
  int lwork = 0, hinfo = 0;
  cudaError_t e = cudaMalloc(&dA, sizeof(double) * n * n);
  if (e == cudaSuccess) e = cudaMalloc(&dW, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&info, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dA, H.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error("plan: device allocation/copy failed: %s", cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? TS_ERR_NO_MEMORY : TS_ERR_CUDA;
  }
  if (st == TS_OK &&
      cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, &lwork) !=
          CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd_bufferSize failed");
    st = TS_ERR_CUDA;
  }
  if (st == TS_OK && cudaMalloc(&work, sizeof(double) * (lwork > 0 ? lwork : 1)) != cudaSuccess) {
    set_error("plan: workspace allocation failed");
    st = TS_ERR_NO_MEMORY;
  }
  if (st == TS_OK &&
      cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, work, lwork, info) !=
          CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd failed");
    st = TS_ERR_CUDA;
  }
  if (st == TS_OK) {
    lam.resize(n);
    Qcol.resize((size_t)n * n);
    e = cudaMemcpyAsync(lam.data(), dW, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Qcol.data(), dA, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("plan: eigendecomposition readback failed: %s", cudaGetErrorString(e));
      st = TS_ERR_CUDA;
    } else if (hinfo != 0) {
      set_error("syevd returned info = %d", hinfo);
      st = TS_ERR_CUDA;
    }
  }
  cudaFree(dA);
  cudaFree(dW);
  cudaFree(work);
  cudaFree(info);
  cusolverDnDestroy(h);
  return st;
}

template <typename T>
ts_status upload(T** dst, const T* src, size_t count, ts_plan* p, cudaStream_t s) {
  TS_CHECK_CUDA(cudaMalloc((void**)dst, sizeof(T) * count));
  p->bytes += (long long)(sizeof(T) * count);
  TS_CHECK_CUDA(cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return TS_OK;
}

}  // namespace

void plan_free(ts_plan* p) {
  if (!p) return;
  for (int k = 0; k < p->d; ++k) {
    if (p->owner[k] != k) continue;
    cudaFree(p->S[k]);
    cudaFree(p->St[k]);
    cudaFree(p->lam[k]);
    cudaFree(p->lamf[k]);
    cudaFree(p->Sf32[k]);
    cudaFree(p->Stf32[k]);
    for (int q = 0; q < NPREC; ++q) {
      cudaFree(p->Bf[q][k]);
      cudaFree(p->Bb[q][k]);
    }
  }
  for (int k = 0; k < p->d; ++k) cudaFree(p->f[k]);  // potential samples are per axis
  delete p;
}

ts_status plan_create(const ts_plan_desc* desc, unsigned mask, cudaStream_t s, ts_plan** out) {
  ts_plan* p = new ts_plan();
  TS_CHECK_CUDA(cudaGetDevice(&p->device));
  p->d = desc->d;
  p->N = 1;
  p->precision_mask = mask | 1u;
  for (int k = 0; k < p->d; ++k) {
    p->n[k] = desc->n[k];
    p->L[k] = desc->L[k];
    p->N *= desc->n[k];
    if (desc->n[k] > p->nmax) p->nmax = desc->n[k];
  }
  ts_status st = TS_OK;
  for (int k = 0; k < p->d && st == TS_OK; ++k) {
    const int n = p->n[k];
    st = upload(&p->f[k], desc->f[k], (size_t)n, p, s);
    if (st != TS_OK) break;
    // Share the decomposition with an earlier identical axis.
    int same = -1;
    for (int j = 0; j < k; ++j)
      if (p->n[j] == n && p->L[j] == p->L[k] && std::memcmp(desc->f[j], desc->f[k], sizeof(double) * n) == 0) {
        same = p->owner[j];
        break;
      }
    if (same >= 0) {
      p->owner[k] = same;
      p->S[k] = p->S[same];
      p->St[k] = p->St[same];
      p->lam[k] = p->lam[same];
      p->lamf[k] = p->lamf[same];
      p->lam_host[k] = p->lam_host[same];
      p->S_host[k] = p->S_host[same];
      continue;
    }
    p->owner[k] = k;
    const double h = 2.0 * p->L[k] / (n + 1);
    const double ih2 = 1.0 / (h * h);
    std::vector<double> H((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
      H[(size_t)i * n + i] = 2.0 * ih2 + desc->f[k][i];
      if (i > 0) H[(size_t)i * n + i - 1] = -ih2;
      if (i + 1 < n) H[(size_t)i * n + i + 1] = -ih2;
    }
    std::vector<double> Qcol;
    st = eig_on_device(n, H, p->lam_host[k], Qcol, s);
    if (st != TS_OK) break;
    // Qcol is column-major: Qcol[i + n j] = S[i][j], i.e. the row-major S^T.
    std::vector<double> S((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) S[(size_t)i * n + j] = Qcol[(size_t)i + (size_t)n * j];
    p->S_host[k] = S;
    st = upload(&p->S[k], S.data(), S.size(), p, s);
    if (st == TS_OK) st = upload(&p->St[k], Qcol.data(), Qcol.size(), p, s);
    if (st == TS_OK) st = upload(&p->lam[k], p->lam_host[k].data(), (size_t)n, p, s);
    std::vector<float> lf(p->lam_host[k].begin(), p->lam_host[k].end());
    if (st == TS_OK) st = upload(&p->lamf[k], lf.data(), (size_t)n, p, s);
    if (st == TS_OK) {
      cudaError_t e = cudaStreamSynchronize(s);  // host vectors go out of scope
      if (e != cudaSuccess) {
        set_error("plan upload failed: %s", cudaGetErrorString(e));
        st = TS_ERR_CUDA;
      }
    }
  }
  for (int q = 1; q < NPREC && st == TS_OK; ++q) {
    if (!(p->precision_mask & (1u << q))) continue;
    st = q == TS_FP32 ? build_small_tables(p, s) : build_split_tables(p, (ts_precision)q, s);
  }
  if (st == TS_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("plan creation failed: %s", cudaGetErrorString(e));
      st = TS_ERR_CUDA;
    }
  }
  if (st != TS_OK) {
    plan_free(p);
    *out = nullptr;
    return st;
  }
  *out = p;
  return TS_OK;
}

}  // namespace ts
