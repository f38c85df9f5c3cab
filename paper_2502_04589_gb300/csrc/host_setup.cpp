// Host-side setup of the multigrid hierarchy: CSR validation, transpose, sparse
// products (Galerkin coarse operators P^T A P for nested spaces, paper §2.2) and a dense
// SPD inverse for the coarsest multigrid level.  Runs once in pase_setup.
#include <math.h>
#include <omp.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <set>
#include <utility>

#include "pase_internal.h"

namespace pase {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
const char* last_error_cstr() { return g_last_error.c_str(); }

// The dynamic shared-memory limit is a per-device property of a kernel: raise it once
// per (device, kernel), safely from several host threads.
int ensure_max_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  PASE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, func})) return PASE_OK;
  PASE_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({dev, func});
  return PASE_OK;
}

int csr_from_abi(const pase_csr* in, HostCSR& out, const char* name) {
  if (!in) return fail(PASE_ERR_INVALID_ARG, std::string(name) + ": null matrix");
  if (in->nrows < 0 || in->ncols < 0 || in->nnz < 0 || in->nrows > INT32_MAX || in->ncols > INT32_MAX)
    return fail(PASE_ERR_INVALID_ARG, std::string(name) + ": bad dimensions");
  if (in->nrows > 0 && (!in->rowptr || (in->nnz > 0 && (!in->colind || !in->val))))
    return fail(PASE_ERR_INVALID_ARG, std::string(name) + ": null array");
  out.nrows = in->nrows;
  out.ncols = in->ncols;
  out.rowptr.resize(in->nrows + 1);
  out.col.resize(in->nnz);
  out.val.resize(in->nnz);
  if (in->on_device) {
    PASE_CUDA(cudaMemcpy(out.rowptr.data(), in->rowptr, sizeof(int64_t) * (in->nrows + 1), cudaMemcpyDeviceToHost));
    if (in->nnz) {
      PASE_CUDA(cudaMemcpy(out.col.data(), in->colind, sizeof(int32_t) * in->nnz, cudaMemcpyDeviceToHost));
      PASE_CUDA(cudaMemcpy(out.val.data(), in->val, sizeof(double) * in->nnz, cudaMemcpyDeviceToHost));
    }
  } else {
    memcpy(out.rowptr.data(), in->rowptr, sizeof(int64_t) * (in->nrows + 1));
    if (in->nnz) {
      memcpy(out.col.data(), in->colind, sizeof(int32_t) * in->nnz);
      memcpy(out.val.data(), in->val, sizeof(double) * in->nnz);
    }
  }
  if (out.rowptr[0] != 0 || out.rowptr[in->nrows] != in->nnz)
    return fail(PASE_ERR_BAD_CSR, std::string(name) + ": rowptr[0] != 0 or rowptr[n] != nnz");
  int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
  for (int64_t i = 0; i < in->nrows; ++i) {
    int64_t a = out.rowptr[i], b = out.rowptr[i + 1];
    if (b < a) {
      bad |= 1;
      continue;
    }
    for (int64_t k = a; k < b; ++k) {
      int32_t c = out.col[k];
      if (c < 0 || c >= in->ncols) bad |= 2;
      if (k > a && c <= out.col[k - 1]) bad |= 4;
      if (!isfinite(out.val[k])) bad |= 8;
    }
  }
  if (bad & 1) return fail(PASE_ERR_BAD_CSR, std::string(name) + ": rowptr not monotone");
  if (bad & 2) return fail(PASE_ERR_BAD_CSR, std::string(name) + ": column index out of range");
  if (bad & 4) return fail(PASE_ERR_BAD_CSR, std::string(name) + ": columns not strictly ascending");
  if (bad & 8) return fail(PASE_ERR_NAN, std::string(name) + ": non-finite value");
  return PASE_OK;
}

bool same_pattern(const HostCSR& a, const HostCSR& b) {
  return a.nrows == b.nrows && a.ncols == b.ncols && a.rowptr == b.rowptr && a.col == b.col;
}

HostCSR csr_transpose(const HostCSR& a) {
  HostCSR t;
  t.nrows = a.ncols;
  t.ncols = a.nrows;
  t.rowptr.assign(t.nrows + 1, 0);
  for (int64_t k = 0; k < a.nnz(); ++k) t.rowptr[a.col[k] + 1]++;
  for (int64_t i = 0; i < t.nrows; ++i) t.rowptr[i + 1] += t.rowptr[i];
  t.col.resize(a.nnz());
  t.val.resize(a.nnz());
  std::vector<int64_t> next(t.rowptr.begin(), t.rowptr.end() - 1);
  for (int64_t i = 0; i < a.nrows; ++i)  // rows in order -> columns of t sorted
    for (int64_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
      int64_t p = next[a.col[k]]++;
      t.col[p] = (int32_t)i;
      t.val[p] = a.val[k];
    }
  return t;
}

// Row-by-row (Gustavson) sparse product with a dense per-thread accumulator.
HostCSR csr_multiply(const HostCSR& a, const HostCSR& b) {
  HostCSR c;
  c.nrows = a.nrows;
  c.ncols = b.ncols;
  c.rowptr.assign(c.nrows + 1, 0);
  const int nt = omp_get_max_threads();
  // symbolic
  {
    std::vector<std::vector<int64_t>> mark(nt, std::vector<int64_t>(b.ncols, -1));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < a.nrows; ++i) {
      auto& mk = mark[omp_get_thread_num()];
      int64_t cnt = 0;
      for (int64_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
        int32_t j = a.col[k];
        for (int64_t q = b.rowptr[j]; q < b.rowptr[j + 1]; ++q)
          if (mk[b.col[q]] != i) {
            mk[b.col[q]] = i;
            ++cnt;
          }
      }
      c.rowptr[i + 1] = cnt;
    }
  }
  for (int64_t i = 0; i < c.nrows; ++i) c.rowptr[i + 1] += c.rowptr[i];
  c.col.resize(c.rowptr[c.nrows]);
  c.val.resize(c.rowptr[c.nrows]);
  {
    std::vector<std::vector<double>> acc(nt, std::vector<double>(b.ncols, 0.0));
    std::vector<std::vector<int64_t>> mark(nt, std::vector<int64_t>(b.ncols, -1));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < a.nrows; ++i) {
      int t = omp_get_thread_num();
      auto& mk = mark[t];
      auto& ac = acc[t];
      int64_t p = c.rowptr[i];
      for (int64_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
        int32_t j = a.col[k];
        double av = a.val[k];
        for (int64_t q = b.rowptr[j]; q < b.rowptr[j + 1]; ++q) {
          int32_t cc = b.col[q];
          if (mk[cc] != i) {
            mk[cc] = i;
            ac[cc] = 0.0;
            c.col[p++] = cc;
          }
          ac[cc] += av * b.val[q];
        }
      }
      std::sort(c.col.begin() + c.rowptr[i], c.col.begin() + c.rowptr[i + 1]);
      for (int64_t q = c.rowptr[i]; q < c.rowptr[i + 1]; ++q) c.val[q] = ac[c.col[q]];
    }
  }
  return c;
}

HostCSR csr_galerkin(const HostCSR& P, const HostCSR& A) {
  HostCSR AP = csr_multiply(A, P);
  HostCSR PT = csr_transpose(P);
  HostCSR C = csr_multiply(PT, AP);
  // symmetrise exactly: the product of a symmetric A is symmetric up to rounding
  HostCSR CT = csr_transpose(C);
  if (same_pattern(C, CT))
    for (int64_t k = 0; k < C.nnz(); ++k) C.val[k] = 0.5 * (C.val[k] + CT.val[k]);
  return C;
}

// Cholesky A = L L^T (row-major dense), then inv = L^-T L^-1.
bool dense_spd_inverse(const HostCSR& a, std::vector<double>& inv) {
  const int64_t n = a.nrows;
  std::vector<double> L(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) L[i * n + a.col[k]] = a.val[k];
  for (int64_t j = 0; j < n; ++j) {
    double d = L[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    L[j * n + j] = d;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double s = L[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / d;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) L[i * n + j] = 0.0;
  // columns of L^-1 by forward substitution: Linv[:, c]
  std::vector<double> Linv(n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) s -= L[i * n + k] * Linv[k * n + c];
      Linv[i * n + c] = s / L[i * n + i];
    }
  }
  inv.assign(n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int64_t k = i; k < n; ++k) s += Linv[k * n + i] * Linv[k * n + j];
      inv[i * n + j] = s;
      inv[j * n + i] = s;
    }
  return true;
}

}  // namespace pase
